// Gradient d logL / d theta (hand-written adjoint of the forward kernels).
//
// logL = -(chi2_pix + chi2_dyn + chi2_tmd)/2 (Eq. chi_general).  The adjoint runs:
//  * lensing: k_conv leaves r_o = mask (d_o - m_o)/sigma_o^2 = d logL/d m_o; k_conv_adj
//    correlates it with the PSF (the transpose of the blurring) into d logL / d img_p;
//    k_image_grad propagates that through every sub-pixel with forward-mode duals over
//    the 8 lens parameters (EPL series, shear) plus analytic Sersic partials for the
//    source (I_e, R_e, n, centre) and lens light (I_e, R_e).
//  * dynamics: k_jam_fg repeats the JAM pair sum while also keeping dV/dx'^2, dV/dy'^2
//    per sky point; k_kin_adj turns the bin adjoints of chi2_dyn (v = sqrt(N/D)) into
//    per-point weights g_N, g_D through the binning-after-PSF operator W and adds the
//    point-coordinate terms (x_c, y_c, phi) and the tracer-amplitude adjoints;
//    k_jam_adj (one thread per table entry, sky points streamed through shared memory)
//    sums the adjoints of each entry (Q0, Q1, a_y); k_grad_chain carries them through the
//    table formula, deprojection (App. A), BH mass and the 1-D MGE (Sect. 3.2) to theta,
//    and adds the delay term by duals through the FP64 lens model.
// The MGE and table quantities are recomputed here, never stored from the forward pass.
#include <algorithm>

#include "cplx.cuh"
#include "dual.cuh"
#include "glad_internal.cuh"
#include "grad_ws.cuh"
#include "jam_common.cuh"
#include "lensmath.cuh"

namespace {

constexpr float LN2F = 0.6931471805599453f;
constexpr double LN2D = 0.6931471805599453;

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void load_lensp(const LensP *src, LensP &dst) {
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(LensP) / 4); i += blockDim.x) d[i] = s[i];
}

// ------------------------------------------------------------------ lensing adjoint

// d logL / d img_p = sum_o r_o P(o - p): correlation of the residual weights with the PSF
__global__ void __launch_bounds__(CONV_TX *CONV_TY) k_conv_adj(const SysDev *__restrict__ sysv,
                                                               const int *__restrict__ sys_id,
                                                               WsDev ws, GradWs g, int max_pix) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int ntx = (S.nx + CONV_TX - 1) / CONV_TX;
  const int nty = (S.ny + CONV_TY - 1) / CONV_TY;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  const int K = S.psf_k, h = (K - 1) / 2;
  const int W = CONV_TX + 2 * h, H = CONV_TY + 2 * h;
  extern __shared__ float sm[];
  float *tile = sm;
  float *psf = sm + H * W;
  const int tid = threadIdx.y * CONV_TX + threadIdx.x;
  const int i0 = ty * CONV_TY - h, j0 = tx * CONV_TX - h;
  const float *r = g.resid + (size_t)b * max_pix;
  for (int e = tid; e < H * W; e += CONV_TX * CONV_TY) {
    const int li = e / W, lj = e - li * W;
    const int gi = i0 + li, gj = j0 + lj;
    tile[e] = (gi >= 0 && gi < S.ny && gj >= 0 && gj < S.nx) ? r[gi * S.nx + gj] : 0.0f;
  }
  for (int e = tid; e < K * K; e += CONV_TX * CONV_TY) psf[e] = S.psf[e];
  __syncthreads();
  const int pi = ty * CONV_TY + threadIdx.y, pj = tx * CONV_TX + threadIdx.x;
  if (pi >= S.ny || pj >= S.nx) return;
  // o = p + (a - h, c - h); tile row of residual row rr is rr - i0
  float acc = 0.0f;
  for (int a = 0; a < K; ++a) {
    const float *trow = tile + (threadIdx.y + a) * W + threadIdx.x;
    const float *prow = psf + a * K;
    for (int c = 0; c < K; ++c) acc = fmaf(prow[c], trow[c], acc);
  }
  g.gpix[(size_t)b * max_pix + pi * S.nx + pj] = acc;
}

typedef Dual<8, float> D8;  // tangents: theta_E, gamma', q, phi, x_c, y_c, gamma_ext, phi_ext

// Sersic value and its partials: I = Ie exp(-bn (w - 1)), w = (R2)^(ninv/2), R2 = (R/Re)^2
struct SersicD {
  float I, dI_dR2, w;
};
__device__ __forceinline__ SersicD sersic_d(float R2, float Ie, float ninv, float bn) {
  SersicD s;
  s.w = exp2f(0.5f * ninv * log2f(R2));
  s.I = Ie * expf(-bn * (s.w - 1.0f));
  s.dI_dR2 = R2 > 1e-30f ? -s.I * bn * s.w * ninv * 0.5f / R2 : 0.0f;
  return s;
}

#define NGL 16  // lensing parameters theta[0..14] and lambda_int (theta[20]) in slot 15

__global__ void __launch_bounds__(LENS_THREADS) k_image_grad(const SysDev *__restrict__ sysv,
                                                             const int *__restrict__ sys_id,
                                                             WsDev ws, GradWs gw, int max_pix,
                                                             double *grad) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.mass_class != 0) return;  // composite samples: k_image_grad_comp
  const int p = blockIdx.x * LENS_THREADS + threadIdx.x;
  __shared__ LensP L;
  __shared__ float red[LENS_THREADS / 32][NGL];
  load_lensp(&ws.lp[b], L);
  __syncthreads();
  float acc[NGL];
#pragma unroll
  for (int i = 0; i < NGL; ++i) acc[i] = 0.0f;
  if (p < S.npix) {
    const int i = p / S.nx, j = p - i * S.nx;
    const int ss = S.ss;
    const float pix = S.pix;
    const float wpix = gw.gpix[(size_t)b * max_pix + p] / (float)(ss * ss);
    const float x0 = (j - 0.5f * (S.nx - 1)) * pix;
    const float y0 = (i - 0.5f * (S.ny - 1)) * pix;
    D8 cphi(L.cphi), sphi(L.sphi), q = D8::var(L.q, 2), t = D8::var(L.t, 1);
    cphi.d[3] = -L.sphi;
    sphi.d[3] = L.cphi;
    D8 pref(L.pref);
    pref.d[0] = L.pref_d[0];
    pref.d[1] = L.pref_d[1];
    pref.d[2] = L.pref_d[2];
    D8 g1(L.g1), g2(L.g2);
    g1.d[6] = L.c2pe;
    g1.d[7] = -2.0f * L.gext * L.s2pe;
    g2.d[6] = L.s2pe;
    g2.d[7] = 2.0f * L.gext * L.c2pe;
    for (int my = 0; my < ss; ++my) {
      const float y = y0 + ((my + 0.5f) / ss - 0.5f) * pix;
      for (int mx = 0; mx < ss; ++mx) {
        const float x = x0 + ((mx + 0.5f) / ss - 0.5f) * pix;
        D8 dx(x - L.xc), dy(y - L.yc);
        dx.d[4] = -1.0f;
        dy.d[5] = -1.0f;
        const D8 xp = cphi * dx + sphi * dy, yp = cphi * dy - sphi * dx;
        // EPL deflection, Tessore & Metcalf series, with tangents
        // at the exact centre alpha is taken as 0 with zero tangents (as in k_image)
        const bool at0 = !(q.v * q.v * xp.v * xp.v + yp.v * yp.v > 0.0f);
        const D8 R = at0 ? D8(1.0f) : dsqrt(q * q * xp * xp + yp * yp);
        const D8 iR = 1.0f / R;
        const D8 wr = q * xp * iR, wi = yp * iR;
        const D8 w2r = wr * wr - wi * wi, w2i = 2.0f * wr * wi;
        D8 omr = wr, omi = wi, Sr = wr, Si = wi;
        for (int n = 0; n < L.nterms; ++n) {
          D8 rr(L.rho[n]);
          rr.d[1] = L.drho_t[n];
          rr.d[2] = L.drho_q[n];
          const D8 nr = rr * (w2r * omr - w2i * omi);
          const D8 ni = rr * (w2r * omi + w2i * omr);
          omr = nr;
          omi = ni;
          Sr = Sr + omr;
          Si = Si + omi;
        }
        const D8 amp = at0 ? D8(0.0f) : pref * dexp2((1.0f - t) * dlog2(R));
        const D8 apx = amp * Sr, apy = amp * Si;
        D8 ax = cphi * apx - sphi * apy;
        D8 ay = sphi * apx + cphi * apy;
        ax = ax + g1 * dx + g2 * dy;
        ay = ay + g2 * dx - g1 * dy;
        for (int k = 0; k < S.n_sis; ++k) {
          const float te = (float)S.sis[3 * k];
          const float sx = x - (float)S.sis[3 * k + 1], sy = y - (float)S.sis[3 * k + 2];
          const float r2 = sx * sx + sy * sy;
          const float ir = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
          ax.v += te * sx * ir;
          ay.v += te * sy * ir;
        }
        // internal mass sheet: lambda x galaxy + (1 - lambda) u (dx, dy); the sheet follows the
        // lens centre (tangents 4, 5 through dx, dy); d alpha / d lambda = galaxy - u (dx, dy)
        float dax_dl = 0.0f, day_dl = 0.0f;
        if (L.sheet) {
          D8 u(1.0f);
          if (L.sheet == 1) {
            const D8 R2 = dx * dx + dy * dy;
            const D8 Qc = dsqrt(R2 + L.sh_rc2), Qt = dsqrt(R2 + L.sh_rt2);
            u = (2.0f * L.sh_rc * L.sh_rt) * (1.0f + (L.sh_rc + L.sh_rt) / (Qc + Qt)) /
                ((L.sh_rc + Qc) * (L.sh_rt + Qt));
          }
          dax_dl = ax.v - u.v * dx.v;
          day_dl = ay.v - u.v * dy.v;
          const D8 om = (1.0f - L.lam) * u;
          ax = L.lam * ax + om * dx;
          ay = L.lam * ay + om * dy;
        }
        // source at beta: d beta / d theta_i = -d alpha / d theta_i (i < 8); centre: -1
        const float bx = x - ax.v - L.src_x, by = y - ay.v - L.src_y;
        const float cs = S.src_cphi, sn = S.src_sphi, iq2 = 1.0f / (S.src_q * S.src_q);
        const float xs = cs * bx + sn * by, ys = -sn * bx + cs * by;
        const float Re2i = L.src_Rei * L.src_Rei;
        const float Rs2 = (xs * xs + ys * ys * iq2) * Re2i;
        const SersicD sd = sersic_d(Rs2, L.src_Ie, L.src_ninv, L.src_bn);
        const float dI_dbx = sd.dI_dR2 * Re2i * 2.0f * (xs * cs - ys * iq2 * sn);
        const float dI_dby = sd.dI_dR2 * Re2i * 2.0f * (xs * sn + ys * iq2 * cs);
        float gsub[NGL];
#pragma unroll
        for (int k = 0; k < 8; ++k) gsub[k] = -(dI_dbx * ax.d[k] + dI_dby * ay.d[k]);
        gsub[8] = sd.I / L.src_Ie;
        gsub[9] = -sd.dI_dR2 * 2.0f * Rs2 / L.src_Rei * Re2i;  // dR2/dRe = -2 R2 / Re
        {
          // d/dn: bn(n) and w = (R/Re)^(1/n)
          const float lnr = Rs2 > 1e-30f ? 0.5f * logf(Rs2) : 0.0f;
          const float dw_dn = -sd.w * lnr * L.src_ninv * L.src_ninv;
          gsub[10] = sd.I * (-L.src_bnp * (sd.w - 1.0f) - L.src_bn * dw_dn);
        }
        gsub[11] = -dI_dbx;
        gsub[12] = -dI_dby;
        gsub[13] = 0.0f;
        gsub[14] = 0.0f;
        gsub[15] = -(dI_dbx * dax_dl + dI_dby * day_dl);
        // lens light: depends on phi, x_c, y_c through (x', y') and on I_e, R_e of component 0
        for (int c = 0; c < S.n_lcomp; ++c) {
          const float Re2 = L.ll_Rei[c] * L.ll_Rei[c];
          const float R2 = (xp.v * xp.v + yp.v * yp.v * L.ll_qi2[c]) * Re2;
          const SersicD ld = sersic_d(R2, L.ll_Ie[c], L.ll_ninv[c], L.ll_bn[c]);
          const float dxp = ld.dI_dR2 * Re2 * 2.0f * xp.v;
          const float dyp = ld.dI_dR2 * Re2 * 2.0f * yp.v * L.ll_qi2[c];
#pragma unroll
          for (int k = 3; k < 6; ++k) gsub[k] += dxp * xp.d[k] + dyp * yp.d[k];
          if (c == 0) {
            gsub[13] = ld.I / L.ll_Ie[0];
            gsub[14] = -ld.dI_dR2 * 2.0f * R2 / L.ll_Rei[0] * Re2;
          }
        }
#pragma unroll
        for (int k = 0; k < NGL; ++k) acc[k] = fmaf(wpix, gsub[k], acc[k]);
      }
    }
  }
  // block reduction, then one FP64 atomic per parameter per block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NGL; ++k) {
    float v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NGL) {
    double s = 0.0;
    for (int w = 0; w < LENS_THREADS / 32; ++w) s += (double)red[w][threadIdx.x];
    const int t = threadIdx.x < 15 ? threadIdx.x : 20;
    if (s != 0.0) atomicAdd(&grad[(size_t)b * GLAD_NTHETA + t], s);
  }
}

// Composite class (Sect. 3.3): the same adjoint with duals over the 12 parameters the ray
// shooting depends on, tangents 0..7 = theta 0..7 (kappa_s, r_s, q of the halo, phi, x_c, y_c,
// shear), 8 = theta 13 (I0), 9 = theta 14 (w_t), 10 = theta 17 (Upsilon_*), 11 = theta 18 (f_BH);
// the halo's CSEs, the Chameleons' softened isothermal pairs and the black-hole Gaussian in dual
// arithmetic; the Chameleon lens light and the Sersic source by analytic partials.
typedef Dual<12, float> D12;
#define NGC 18  // theta 0..14, then lambda_int (20), Upsilon_* (17), f_BH (18)

__device__ __forceinline__ void nie_d12(const D12 &x, const D12 &y, const D12 &A, const D12 &s, float q,
                                        float e, float sg, D12 &ax, D12 &ay) {
  if (e > 1e-3f) {
    const D12 ps = dsqrt(q * q * (s * s + x * x) + y * y);
    const D12 b = (2.0f * q / e) * A;
    ax = ax + sg * (b * datan(e * x / (ps + s)));
    ay = ay + sg * (b * datanh(e * y / (ps + (q * q) * s)));
  } else {
    const D12 fac = 2.0f * A / (dsqrt(x * x + y * y + s * s) + s);
    ax = ax + sg * (fac * x);
    ay = ay + sg * (fac * y);
  }
}

__global__ void __launch_bounds__(LENS_THREADS) k_image_grad_comp(const SysDev *__restrict__ sysv,
                                                                  const int *__restrict__ sys_id,
                                                                  WsDev ws, GradWs gw, int max_pix,
                                                                  double *grad) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.mass_class != 1) return;
  const int p = blockIdx.x * LENS_THREADS + threadIdx.x;
  __shared__ LensP L;
  __shared__ float red[LENS_THREADS / 32][NGC];
  load_lensp(&ws.lp[b], L);
  __syncthreads();
  float acc[NGC];
#pragma unroll
  for (int i = 0; i < NGC; ++i) acc[i] = 0.0f;
  if (p < S.npix) {
    const int i = p / S.nx, j = p - i * S.nx;
    const int ss = S.ss;
    const float pix = S.pix;
    const float wpix = gw.gpix[(size_t)b * max_pix + p] / (float)(ss * ss);
    const float x0 = (j - 0.5f * (S.nx - 1)) * pix;
    const float y0 = (i - 0.5f * (S.ny - 1)) * pix;
    D12 cphi(L.cphi), sphi(L.sphi);
    cphi.d[3] = -L.sphi;
    sphi.d[3] = L.cphi;
    D12 g1(L.g1), g2(L.g2);
    g1.d[6] = L.c2pe;
    g1.d[7] = -2.0f * L.gext * L.s2pe;
    g2.d[6] = L.s2pe;
    g2.d[7] = 2.0f * L.gext * L.c2pe;
    D12 ups(L.ups);  // Upsilon_* L_scale, d/d Upsilon_* = L_scale
    ups.d[10] = (float)S.L_scale;
    D12 bhM(L.bh_M);
    bhM.d[8] = L.bh_dM[0];
    bhM.d[9] = L.bh_dM[1];
    bhM.d[10] = L.bh_dM[2];
    bhM.d[11] = L.bh_dM[3];
    const D12 hq = D12::var(L.h_q, 2);
    const D12 ks = D12::var(L.h_ks, 0), rs = D12::var(L.h_rs, 1);
    for (int my = 0; my < ss; ++my) {
      const float y = y0 + ((my + 0.5f) / ss - 0.5f) * pix;
      for (int mx = 0; mx < ss; ++mx) {
        const float x = x0 + ((mx + 0.5f) / ss - 0.5f) * pix;
        D12 dx(x - L.xc), dy(y - L.yc);
        dx.d[4] = -1.0f;
        dy.d[5] = -1.0f;
        const D12 xp = cphi * dx + sphi * dy, yp = cphi * dy - sphi * dx;
        D12 fx(0.0f), fy(0.0f);
        // baryons: Upsilon L_scale x each Chameleon's pair of softened isothermal ellipsoids
        for (int c = 0; c < S.n_lcomp && c < 4; ++c) {
          D12 A = L.li_A[c] * ups;  // Upsilon_* L_scale I0 / (1 + q)
          if (c == 0) A.d[8] = ups.v / (1.0f + L.ch_q[0]);
          D12 st(L.ch_st[c]);
          if (c == 0) st.d[9] = 2.0f / (1.0f + L.ch_q[c]);
          nie_d12(xp, yp, A, D12(L.ch_sc[c]), L.ch_q[c], L.ch_e[c], 1.0f, fx, fy);
          nie_d12(xp, yp, A, st, L.ch_q[c], L.ch_e[c], -1.0f, fx, fy);
        }
        // halo: CSE i with amplitude kappa_s a_i r_s^3 and core s_i r_s, axis ratio q of the halo
        {
          const D12 q2 = hq * hq, e2 = 1.0f - q2;
          const D12 base = q2 * xp * xp + yp * yp, ex2 = e2 * xp * xp;
          D12 hx(0.0f), hy(0.0f);
          for (int k = 0; k < GLAD_N_CSE; ++k) {
            if (L.cse_a3[k] == 0.0f) continue;
            const float s1 = L.cse_sc[k] / L.h_rs;  // core in units of r_s
            const D12 sc = s1 * rs;
            const D12 amp = ks * (L.cse_a3[k] / (L.h_rs * L.h_rs * L.h_rs)) * rs * rs * rs;
            const D12 ps = dsqrt(base + q2 * sc * sc);
            const D12 D = (ps + sc) * (ps + sc) + ex2;
            const D12 w = amp / (sc * ps * D);
            hx = hx + w * (ps + q2 * sc);
            hy = hy + w * (ps + sc);
          }
          fx = fx + 2.0f * hq * xp * hx;
          fy = fy + 2.0f * hq * yp * hy;
        }
        D12 ax = cphi * fx - sphi * fy;
        D12 ay = sphi * fx + cphi * fy;
        if (L.bh_M > 0.0f) {
          // round Gaussian: M h1(t) / (pi 2 sigma^2) (dx, dy), t = R^2 / (2 sigma^2)
          const D12 t = (dx * dx + dy * dy) / L.bh_2s2;
          D12 h1;
          if (t.v < 1e-3f) {
            h1 = 1.0f - 0.5f * t;
          } else {
            const float em = expf(-t.v), hv = -expm1f(-t.v) / t.v;
            h1 = dual_apply(t, hv, (em * (t.v + 1.0f) - 1.0f) / (t.v * t.v));
          }
          const D12 gfac = bhM * h1 / (3.14159265358979f * L.bh_2s2);
          ax = ax + gfac * dx;
          ay = ay + gfac * dy;
        }
        ax = ax + g1 * dx + g2 * dy;
        ay = ay + g2 * dx - g1 * dy;
        for (int k = 0; k < S.n_sis; ++k) {
          const float te = (float)S.sis[3 * k];
          const float sx = x - (float)S.sis[3 * k + 1], sy = y - (float)S.sis[3 * k + 2];
          const float r2 = sx * sx + sy * sy;
          const float ir = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
          ax.v += te * sx * ir;
          ay.v += te * sy * ir;
        }
        float dax_dl = 0.0f, day_dl = 0.0f;
        if (L.sheet) {
          D12 u(1.0f);
          if (L.sheet == 1) {
            const D12 R2 = dx * dx + dy * dy;
            const D12 Qc = dsqrt(R2 + L.sh_rc2), Qt = dsqrt(R2 + L.sh_rt2);
            u = (2.0f * L.sh_rc * L.sh_rt) * (1.0f + (L.sh_rc + L.sh_rt) / (Qc + Qt)) /
                ((L.sh_rc + Qc) * (L.sh_rt + Qt));
          }
          dax_dl = ax.v - u.v * dx.v;
          day_dl = ay.v - u.v * dy.v;
          const D12 om = (1.0f - L.lam) * u;
          ax = L.lam * ax + om * dx;
          ay = L.lam * ay + om * dy;
        }
        // source at beta = theta - alpha
        const float bx = x - ax.v - L.src_x, by = y - ay.v - L.src_y;
        const float cs = S.src_cphi, sn = S.src_sphi, iq2 = 1.0f / (S.src_q * S.src_q);
        const float xs = cs * bx + sn * by, ys = -sn * bx + cs * by;
        const float Re2i = L.src_Rei * L.src_Rei;
        const float Rs2 = (xs * xs + ys * ys * iq2) * Re2i;
        const SersicD sd = sersic_d(Rs2, L.src_Ie, L.src_ninv, L.src_bn);
        const float dI_dbx = sd.dI_dR2 * Re2i * 2.0f * (xs * cs - ys * iq2 * sn);
        const float dI_dby = sd.dI_dR2 * Re2i * 2.0f * (xs * sn + ys * iq2 * cs);
        float gsub[NGC];
#pragma unroll
        for (int k = 0; k < 8; ++k) gsub[k] = -(dI_dbx * ax.d[k] + dI_dby * ay.d[k]);
        gsub[8] = sd.I / L.src_Ie;
        gsub[9] = -sd.dI_dR2 * 2.0f * Rs2 / L.src_Rei * Re2i;
        {
          const float lnr = Rs2 > 1e-30f ? 0.5f * logf(Rs2) : 0.0f;
          const float dw_dn = -sd.w * lnr * L.src_ninv * L.src_ninv;
          gsub[10] = sd.I * (-L.src_bnp * (sd.w - 1.0f) - L.src_bn * dw_dn);
        }
        gsub[11] = -dI_dbx;
        gsub[12] = -dI_dby;
        gsub[13] = -(dI_dbx * ax.d[8] + dI_dby * ay.d[8]);
        gsub[14] = -(dI_dbx * ax.d[9] + dI_dby * ay.d[9]);
        gsub[15] = -(dI_dbx * dax_dl + dI_dby * day_dl);
        gsub[16] = -(dI_dbx * ax.d[10] + dI_dby * ay.d[10]);
        gsub[17] = -(dI_dbx * ax.d[11] + dI_dby * ay.d[11]);
        // Chameleon lens light: li_A [(m^2 + sc^2)^-1/2 - (m^2 + st^2)^-1/2], m^2 = x'^2 + y'^2/q^2
        for (int c = 0; c < S.n_lcomp && c < 4; ++c) {
          const float q = L.ch_q[c], iq2c = 1.0f / (q * q);
          const float m2 = xp.v * xp.v + yp.v * yp.v * iq2c;
          const float rc = rsqrtf(m2 + L.ch_sc[c] * L.ch_sc[c]), rt = rsqrtf(m2 + L.ch_st[c] * L.ch_st[c]);
          const float dIdm2 = -0.5f * L.li_A[c] * (rc * rc * rc - rt * rt * rt);
          const float dxp = dIdm2 * 2.0f * xp.v, dyp = dIdm2 * 2.0f * yp.v * iq2c;
#pragma unroll
          for (int k = 3; k < 6; ++k) gsub[k] += dxp * xp.d[k] + dyp * yp.d[k];
          if (c == 0) {
            gsub[13] += (rc - rt) / (1.0f + q);                                     // d/d I0
            gsub[14] += L.li_A[0] * rt * rt * rt * L.ch_st[0] * 2.0f / (1.0f + q);  // d/d w_t
          }
        }
#pragma unroll
        for (int k = 0; k < NGC; ++k) acc[k] = fmaf(wpix, gsub[k], acc[k]);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    float v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NGC) {
    double s = 0.0;
    for (int w = 0; w < LENS_THREADS / 32; ++w) s += (double)red[w][threadIdx.x];
    const int k = threadIdx.x;
    const int t = k < 15 ? k : (k == 15 ? 20 : (k == 16 ? 17 : 18));
    if (s != 0.0) atomicAdd(&grad[(size_t)b * GLAD_NTHETA + t], s);
  }
}

// ------------------------------------------------------------------ dynamics adjoint

// Launch shape of the derivative pass: 2 points per thread, at least 4 CTAs per SM (64
// registers); measured at B = 64 against 4 points / 3 CTAs (7.45 vs 8.23 ms) and 8 points /
// 2 CTAs (9.81 ms).
#define FG_PTS 2
#define FG_MINB 4

// JAM pair sum with dV/dX and dV/dY per point (X = x'^2, Y = y'^2), plus the same bin
// scatter as the forward kernel so that v_rms and chi2_dyn come out of this pass too.
// Same 2-D sky tiles and exact skipping of entries flushed to zero as the forward kernel
// (FG_PTS points per thread).
__global__ void __launch_bounds__(JAM_THREADS, FG_MINB) k_jam_fg(const SysDev *__restrict__ sysv,
                                                        const int *__restrict__ sys_id, WsDev ws,
                                                        GradWs gw, int max_light, int max_ent,
                                                        int max_bins, int max_sub) {
  constexpr int PTS = FG_PTS, NP = PTS / 2, TH = (JAM_THREADS / JAM_TW) * PTS;
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int tile = blockIdx.x;
  if (S.jam_align != 0 || tile >= jam_tiles(S.nsx, S.nsy, PTS)) return;
  __shared__ JamSmem sm;
  const int tid = threadIdx.x;
  const DynP dp = ws.dp[b];
  const int ntx = (S.nsx + JAM_TW - 1) / JAM_TW;
  const int c0 = (tile % ntx) * JAM_TW, r0 = (tile / ntx) * TH;
  const int c1 = min(c0 + JAM_TW, S.nsx) - 1, r1 = min(r0 + TH, S.nsy) - 1;
  for (int l = tid; l < S.n_bins; l += JAM_THREADS) {
    sm.bnum[l] = 0.0f;
    sm.bden[l] = 0.0f;
  }
  for (int k = tid; k < S.n_light; k += JAM_THREADS) {
    sm.sI0[k] = ws.I0f[(size_t)b * max_light + k];
    sm.scx[k] = S.sb_cx[k];
    sm.scy[k] = S.sb_cy[k];
  }
  float Xmin, Ymin;
  jam_tile_bounds(S, dp, c0, c1, r0, r1, Xmin, Ymin);
  const float Xmax = jam_tile_xmax(S, dp, c0, c1, r0, r1);
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  const float xc = (float)dp.xc, yc = (float)dp.yc;
  const float hx = 0.5f * (S.nsx - 1), hy = 0.5f * (S.nsy - 1);
  const float4 *gt = ws.tab + (size_t)b * max_ent;
  const int n_ent = S.n_ent;
  const int n_chunks = (n_ent + JAM_CHUNK - 1) / JAM_CHUNK;
  const int lane = tid & 31, warp = tid >> 5;
  // Negligible terms as in the forward pass (reference: the full sum at the tile's corners),
  // with the a-posteriori check covering V, dV/dX and dV/dY.
  float lref = 0.0f, lrel = -INFINITY;
  if (ws.neg_mode != 0) {
    float cX[4], cY[4], cv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = ((q & 1 ? c1 : c0) - hx) * S.dsub - xc;
      const float y = ((q & 2 ? r1 : r0) - hy) * S.dsub - yc;
      const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
      cX[q] = xp * xp;
      cY[q] = yp * yp;
      cv[q] = 0.0f;
    }
    for (int e = tid; e < n_ent; e += JAM_THREADS) {
      const float4 c = gt[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        cv[q] = fmaf(fmaf(c.w, cX[q], c.z), jam_ex2(fmaf(c.y, cY[q], c.x * cX[q])), cv[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      for (int off = 16; off > 0; off >>= 1) cv[q] += __shfl_xor_sync(0xffffffffu, cv[q], off);
      if (lane == 0) sm.red[q][warp] = cv[q];
    }
    __syncthreads();
    if (tid == 0) {
      float ref = 3.4e38f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float t = 0.0f;
        for (int w = 0; w < JAM_THREADS / 32; ++w) t += sm.red[q][w];
        ref = fminf(ref, t);
      }
      sm.flag = (ref > 0.0f && ref < 3.4e38f) ? __float_as_int(__log2f(ref)) : 0x7fffffff;
    }
    __syncthreads();
    const int f = sm.flag;
    lref = f == 0x7fffffff ? 0.0f : __int_as_float(f);
    lrel = f == 0x7fffffff ? -INFINITY : -(JAM_REL_MARGIN_GRAD + __log2f((float)max(n_ent, 1)));
  }
  if (tid == 0) {
    sm.tb[0] = Xmin;
    sm.tb[1] = Ymin;
    sm.tb[2] = Xmax;
    sm.tb[3] = lref;
    sm.tb[4] = lrel;
  }
  __syncthreads();
  const int col = c0 + (tid % JAM_TW);
  const int row0 = r0 + (tid / JAM_TW) * PTS;
  float2 X[NP], Y[NP];
  float2 aV[NP], a1[NP], a2[NP], a3[NP];
  double dV[PTS], d1[PTS], d2[PTS], d3[PTS];
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    const int J = min(col, c1), I = min(row0 + i, r1);
    const float x = (J - hx) * S.dsub - xc;
    const float y = (I - hy) * S.dsub - yc;
    const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
    if (i & 1) {
      X[i >> 1].y = xp * xp;
      Y[i >> 1].y = yp * yp;
    } else {
      X[i >> 1].x = xp * xp;
      Y[i >> 1].x = yp * yp;
    }
  }
  const float2 z2 = make_float2(0.f, 0.f);
  const unsigned long long npts = (unsigned long long)(c1 - c0 + 1) * (unsigned long long)(r1 - r0 + 1);
  unsigned long long n_eval = 0;  // evaluations this tile executes (thread 0 keeps the count)
  for (;;) {
#pragma unroll
    for (int i = 0; i < PTS; ++i) dV[i] = d1[i] = d2[i] = d3[i] = 0.0;
#pragma unroll
    for (int p = 0; p < NP; ++p) aV[p] = a1[p] = a2[p] = a3[p] = z2;
    float rv = 0.0f, rx = 0.0f, ry = 0.0f;  // left-out bounds relative to the reference
    JamStager stg;
    stg.count_rel_grad(gt, n_ent, 0, sm.tb, sm.wcount[0], rv, rx, ry);
    __syncthreads();
    stg.write(sm.tab[0], sm.wcount[0], &sm.n_kept[0]);
    __syncthreads();
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int cur = ch & 1;
      const bool more = ch + 1 < n_chunks;
      if (more)
        stg.count_rel_grad(gt, n_ent, (ch + 1) * JAM_CHUNK, sm.tb, sm.wcount[cur ^ 1], rv, rx, ry);
      const float4 *tt = sm.tab[cur];
      const int nk = sm.n_kept[cur];
      n_eval += (unsigned long long)nk * npts;
#pragma unroll 2
      for (int e = 0; e < nk; ++e) {
        const float4 c = tt[e];
        const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y);
        const float2 cz = make_float2(c.z, c.z), cw = make_float2(c.w, c.w);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 arg = __ffma2_rn(cy, Y[p], __fmul2_rn(cx, X[p]));
          const float2 E = make_float2(jam_ex2(arg.x), jam_ex2(arg.y));
          const float2 tv = __fmul2_rn(__ffma2_rn(cw, X[p], cz), E);
          aV[p] = __fadd2_rn(aV[p], tv);
          a1[p] = __ffma2_rn(cw, E, a1[p]);
          a2[p] = __ffma2_rn(cx, tv, a2[p]);
          a3[p] = __ffma2_rn(cy, tv, a3[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        dV[2 * p] += aV[p].x;
        dV[2 * p + 1] += aV[p].y;
        d1[2 * p] += a1[p].x;
        d1[2 * p + 1] += a1[p].y;
        d2[2 * p] += a2[p].x;
        d2[2 * p + 1] += a2[p].y;
        d3[2 * p] += a3[p].x;
        d3[2 * p + 1] += a3[p].y;
        aV[p] = a1[p] = a2[p] = a3[p] = z2;
      }
      __syncthreads();
      if (more) stg.write(sm.tab[cur ^ 1], sm.wcount[cur ^ 1], &sm.n_kept[cur ^ 1]);
      __syncthreads();
    }
    if (lrel == -INFINITY) break;
    // a-posteriori check: the left-out bound of V against the smallest |V| in the tile; those
    // of dV/dX and dV/dY (sums of mixed signs, which can pass through zero) against their
    // largest magnitude in the tile, i.e. below the FP32 rounding of those sums
    float mv = 3.4e38f, mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int i = 0; i < PTS; ++i)
      if (col <= c1 && row0 + i <= r1) {
        mv = fminf(mv, fabsf((float)dV[i]));
        mx = fmaxf(mx, fabsf((float)(d1[i] + LN2D * d2[i])));
        my = fmaxf(my, fabsf((float)(LN2D * d3[i])));
      }
    for (int off = 16; off > 0; off >>= 1) {
      mv = fminf(mv, __shfl_xor_sync(0xffffffffu, mv, off));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, off));
      rv += __shfl_xor_sync(0xffffffffu, rv, off);
      rx += __shfl_xor_sync(0xffffffffu, rx, off);
      ry += __shfl_xor_sync(0xffffffffu, ry, off);
    }
    __shared__ float chk[6][JAM_THREADS / 32];
    if (lane == 0) {
      chk[0][warp] = mv;
      chk[1][warp] = mx;
      chk[2][warp] = my;
      chk[3][warp] = rv;
      chk[4][warp] = rx;
      chk[5][warp] = ry;
    }
    __syncthreads();
    if (tid == 0) {
      float m[3] = {3.4e38f, 0.f, 0.f}, r[3] = {0.f, 0.f, 0.f};
      for (int w = 0; w < JAM_THREADS / 32; ++w) {
        m[0] = fminf(m[0], chk[0][w]);
        m[1] = fmaxf(m[1], chk[1][w]);
        m[2] = fmaxf(m[2], chk[2][w]);
        for (int q = 0; q < 3; ++q) r[q] += chk[3 + q][w];
      }
      bool ok = ws.neg_mode == 1;
      for (int q = 0; q < 3; ++q) ok = ok && (__log2f(r[q]) + lref <= __log2f(m[q]) - JAM_REL_CHECK);
      sm.flag = ok ? 1 : 0;
    }
    __syncthreads();
    const bool ok = sm.flag != 0;
    __syncthreads();
    if (ok) break;
    lrel = -INFINITY;  // sum the tile again with the exact skipping only
    if (tid == 0) sm.tb[4] = -INFINITY;
    __syncthreads();
  }
  if (tid == 0 && ws.evals) atomicAdd(ws.evals, n_eval);
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    if (col > c1 || row0 + i > r1) continue;
    const int s = (row0 + i) * S.nsx + col;
    const float Xi = (i & 1) ? X[i >> 1].y : X[i >> 1].x;
    const float Yi = (i & 1) ? Y[i >> 1].y : Y[i >> 1].x;
    float sb = 0.0f;
    for (int k = 0; k < S.n_light; ++k)
      sb = fmaf(sm.sI0[k], jam_ex2(-fmaf(sm.scy[k], Yi, sm.scx[k] * Xi)), sb);
    const float v = (float)dV[i];
    // coefficients are in log2 units: d/dX 2^(ax X) = ln2 ax 2^(ax X)
    gw.pt[(size_t)b * max_sub + s] =
        make_float4(v, (float)(d1[i] + LN2D * d2[i]), (float)(LN2D * d3[i]), sb);
    for (int e = S.w_off[s]; e < S.w_off[s + 1]; ++e) {
      const int l = S.w_bin[e];
      const float w = S.w_val[e];
      atomicAdd(&sm.bnum[l], w * v);
      atomicAdd(&sm.bden[l], w * sb);
    }
  }
  __syncthreads();
  double *acc_g = ws.binacc + (size_t)b * max_bins * 2;
  for (int l = tid; l < S.n_bins; l += JAM_THREADS) {
    if (sm.bnum[l] != 0.0f) atomicAdd(&acc_g[2 * l], (double)sm.bnum[l]);
    if (sm.bden[l] != 0.0f) atomicAdd(&acc_g[2 * l + 1], (double)sm.bden[l]);
  }
}

// Per sky point: g_N = sum_l W_l gN_l, g_D = sum_l W_l gD_l with gN_l = d logL/d N_l,
// gD_l = d logL/d D_l of v_l = sqrt(N_l/D_l); coordinate and tracer-amplitude adjoints.
__global__ void __launch_bounds__(JAM_THREADS) k_kin_adj(const SysDev *__restrict__ sysv,
                                                         const int *__restrict__ sys_id, WsDev ws,
                                                         GradWs gw, int max_light, int max_bins,
                                                         int max_sub, int max_apts, double *grad) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int tile0 = blockIdx.x * JAM_TILE;
  if (tile0 >= S.n_sub) return;
  __shared__ float gN[GLAD_MAX_BINS], gD[GLAD_MAX_BINS];
  __shared__ float sI0[GLAD_MAX_LIGHT], scx[GLAD_MAX_LIGHT], scy[GLAD_MAX_LIGHT];
  __shared__ float aI0[GLAD_MAX_LIGHT];
  __shared__ float red[JAM_THREADS / 32][3];
  const int tid = threadIdx.x;
  const double *acc = ws.binacc + (size_t)b * max_bins * 2;
  for (int l = tid; l < S.n_bins; l += JAM_THREADS) {
    const double N = acc[2 * l], D = acc[2 * l + 1];
    const double v = sqrt(N / D);
    const double sg = (double)S.v_sig[l];
    const double dv = ((double)S.v_obs[l] - v) / (sg * sg);  // d logL / d v
    gN[l] = (float)(dv / (2.0 * v * D));
    gD[l] = (float)(-dv * v / (2.0 * D));
  }
  for (int k = tid; k < S.n_light; k += JAM_THREADS) {
    sI0[k] = ws.I0f[(size_t)b * max_light + k];
    scx[k] = S.sb_cx[k];
    scy[k] = S.sb_cy[k];
    aI0[k] = 0.0f;
  }
  __syncthreads();
  const DynP dp = ws.dp[b];
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  const float xc = (float)dp.xc, yc = (float)dp.yc;
  const int lane = tid & 31;
  float gphi = 0.0f, gxc = 0.0f, gyc = 0.0f;
  // this thread's points (strided by the block), their coordinates and bin adjoints
  float X[JAM_PTS], Y[JAM_PTS], xpv[JAM_PTS], ypv[JAM_PTS], gnv[JAM_PTS], gdv[JAM_PTS];
  float dsx[JAM_PTS], dsy[JAM_PTS];
#pragma unroll
  for (int i = 0; i < JAM_PTS; ++i) {
    const int s = tile0 + tid + i * JAM_THREADS;
    X[i] = Y[i] = xpv[i] = ypv[i] = gnv[i] = gdv[i] = dsx[i] = dsy[i] = 0.0f;
    if (s >= S.n_sub) continue;
    const int I = s / S.nsx, J = s - I * S.nsx;
    const float x = (J - 0.5f * (S.nsx - 1)) * S.dsub - xc;
    const float y = (I - 0.5f * (S.nsy - 1)) * S.dsub - yc;
    xpv[i] = cphi * x + sphi * y;
    ypv[i] = -sphi * x + cphi * y;
    X[i] = xpv[i] * xpv[i];
    Y[i] = ypv[i] * ypv[i];
    float gn = 0.0f, gd = 0.0f;
    for (int e = S.w_off[s]; e < S.w_off[s + 1]; ++e) {
      const int l = S.w_bin[e];
      const float w = S.w_val[e];
      gn = fmaf(w, gN[l], gn);
      gd = fmaf(w, gD[l], gd);
    }
    gnv[i] = gn;
    gdv[i] = gd;
  }
  // tracer surface brightness derivatives; d logL / d I0_k summed over the warp's points
  // (warp shuffles, one shared atomic per warp and Gaussian)
  for (int k = 0; k < S.n_light; ++k) {
    const float cxk = scx[k], cyk = scy[k], ik = sI0[k];
    float a = 0.0f;
#pragma unroll
    for (int i = 0; i < JAM_PTS; ++i) {
      const float E = ex2(-fmaf(cyk, Y[i], cxk * X[i]));
      a = fmaf(gdv[i], E, a);
      dsx[i] = fmaf(ik * cxk, E, dsx[i]);
      dsy[i] = fmaf(ik * cyk, E, dsy[i]);
    }
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0 && a != 0.0f) atomicAdd(&aI0[k], a);
  }
#pragma unroll
  for (int i = 0; i < JAM_PTS; ++i) {
    const int s = tile0 + tid + i * JAM_THREADS;
    if (s >= S.n_sub) continue;
    const int I = s / S.nsx, J = s - I * S.nsx;
    const float4 pv = gw.pt[(size_t)b * max_sub + s];
    const float gn = gnv[i], gd = gdv[i], xp = xpv[i], yp = ypv[i];
    const float aX = gn * pv.y - gd * LN2F * dsx[i];
    const float aY = gn * pv.z - gd * LN2F * dsy[i];
    // X = x'^2, Y = y'^2; dx'/dphi = y', dy'/dphi = -x'; dx'/dxc = -c, dy'/dxc = s;
    // dx'/dyc = -s, dy'/dyc = -c
    gphi += 2.0f * xp * yp * (aX - aY);
    gxc += aX * (-2.0f * xp * cphi) + aY * (2.0f * yp * sphi);
    gyc += aX * (-2.0f * xp * sphi) + aY * (-2.0f * yp * cphi);
    // position in 16 x 16 point tiles (tile-major), the adjoint's chunk order
    const size_t pos = (size_t)b * max_apts +
                       (size_t)((I >> 4) * S.atx + (J >> 4)) * 256 + (I & 15) * 16 + (J & 15);
    gw.adjpt[2 * pos] = make_float4(X[i], X[i], Y[i], Y[i]);
    gw.adjpt[2 * pos + 1] = make_float4(X[i] * Y[i], X[i] * Y[i], gn, gn);
  }
  const int warp = tid >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    gphi += __shfl_down_sync(0xffffffffu, gphi, off);
    gxc += __shfl_down_sync(0xffffffffu, gxc, off);
    gyc += __shfl_down_sync(0xffffffffu, gyc, off);
  }
  if (lane == 0) {
    red[warp][0] = gphi;
    red[warp][1] = gxc;
    red[warp][2] = gyc;
  }
  __syncthreads();
  if (tid < 3) {
    double s = 0.0;
    for (int w = 0; w < JAM_THREADS / 32; ++w) s += (double)red[w][tid];
    atomicAdd(&grad[(size_t)b * GLAD_NTHETA + 3 + tid], s);  // phi, x_c, y_c = theta[3..5]
  }
  for (int k = tid; k < S.n_light; k += JAM_THREADS)
    if (aI0[k] != 0.0f) atomicAdd(&gw.adjI0[(size_t)b * max_light + k], (double)aI0[k]);
}

#define ADJ_THREADS 256
#define ADJ_PCHUNK 256     // sky points per shared-memory chunk: one 16 x 16 tile

// d logL / d (Q0, Q1, a_y) of each table entry: sums over every sky point of
// g_N(s) E(s) {1, X, (Q0 + Q1 X) Y} with E = 2^(ax X + ay Y).  Each thread owns EPT entries,
// handled as EPT/2 packed pairs against the pre-duplicated point data.  Entries are taken in
// ascending order of p (adj_perm) so that a warp's entries decay alike; a warp skips a
// 16 x 16 point tile for an entry pair when the exponent bound of every lane's pair over the
// tile is below -130 (all those E flush to exactly 0, as in the forward kernel).
template <int EPT>
__global__ void __launch_bounds__(ADJ_THREADS) k_jam_adj(const SysDev *__restrict__ sysv,
                                                         const int *__restrict__ sys_id, WsDev ws,
                                                         GradWs gw, int max_ent, int max_apts) {
  constexpr int NP = EPT / 2;
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int e0 = blockIdx.x * ADJ_THREADS * EPT;
  if (S.jam_align != 0 || e0 >= S.n_ent) return;
  __shared__ float4 pts[2][2 * ADJ_PCHUNK];
  const int tid = threadIdx.x;
  const DynP dp = ws.dp[b];
  // entry pair p of the thread: sorted positions e0 + tid + (2p) * T and e0 + tid + (2p+1) * T
  int ent[EPT];
  float2 ax[NP], ay[NP], s0[NP], sx[NP], sy[NP], sxy[NP];
  double S0[EPT], SX[EPT], SY[EPT], SXY[EPT];
  const float4 *gt = ws.tab + (size_t)b * max_ent;
  const float2 z2 = make_float2(0.f, 0.f);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int o = e0 + tid + k * ADJ_THREADS;
    ent[k] = o < S.n_ent ? S.adj_perm[o] : -1;
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float4 ca = ent[2 * p] >= 0 ? gt[ent[2 * p]] : z4;
    const float4 cb = ent[2 * p + 1] >= 0 ? gt[ent[2 * p + 1]] : z4;
    // padding entries get a hugely negative exponent so that they never keep a tile alive
    ax[p] = make_float2(ent[2 * p] >= 0 ? ca.x : -1e30f, ent[2 * p + 1] >= 0 ? cb.x : -1e30f);
    ay[p] = make_float2(ent[2 * p] >= 0 ? ca.y : -1e30f, ent[2 * p + 1] >= 0 ? cb.y : -1e30f);
    s0[p] = sx[p] = sy[p] = sxy[p] = z2;
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) S0[k] = SX[k] = SY[k] = SXY[k] = 0.0;
  const float4 *gp = gw.adjpt + 2 * (size_t)b * max_apts;
  const int n_chunks = S.n_atile;
  unsigned long long n_eval = 0;  // (entry, point) pairs this thread evaluates
  for (int i = tid; i < 2 * ADJ_PCHUNK; i += ADJ_THREADS) pts[0][i] = gp[i];
  __syncthreads();
  for (int ch = 0; ch < n_chunks; ++ch) {
    const int cur = ch & 1;
    if (ch + 1 < n_chunks) {
      const int base = 2 * (ch + 1) * ADJ_PCHUNK;
      for (int i = tid; i < 2 * ADJ_PCHUNK; i += ADJ_THREADS) pts[cur ^ 1][i] = gp[base + i];
    }
    // which entry pairs this warp needs on this tile
    float Xm, Ym;
    {
      const int c0 = (ch % S.atx) * 16, r0 = (ch / S.atx) * 16;
      jam_tile_bounds(S, dp, c0, min(c0 + 15, S.nsx - 1), r0, min(r0 + 15, S.nsy - 1), Xm, Ym);
    }
    bool need[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const bool mine = fmaf(ay[p].x, Ym, ax[p].x * Xm) >= JAM_SKIP_LOG2 ||
                        fmaf(ay[p].y, Ym, ax[p].y * Xm) >= JAM_SKIP_LOG2;
      need[p] = __any_sync(0xffffffffu, mine);
    }
    const float4 *pp = pts[cur];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      if (!need[p]) continue;  // warp-uniform
      n_eval += ((ent[2 * p] >= 0) + (ent[2 * p + 1] >= 0)) * ADJ_PCHUNK;
#pragma unroll 4
      for (int i = 0; i < ADJ_PCHUNK; ++i) {
        const float4 A = pp[2 * i], Bq = pp[2 * i + 1];  // (X, X, Y, Y), (XY, XY, g, g)
        const float2 X2 = make_float2(A.x, A.y), Y2 = make_float2(A.z, A.w);
        const float2 XY2 = make_float2(Bq.x, Bq.y), G2 = make_float2(Bq.z, Bq.w);
        const float2 arg = __ffma2_rn(ay[p], Y2, __fmul2_rn(ax[p], X2));
        const float2 tg = __fmul2_rn(G2, make_float2(jam_ex2(arg.x), jam_ex2(arg.y)));
        s0[p] = __fadd2_rn(s0[p], tg);
        sx[p] = __ffma2_rn(tg, X2, sx[p]);
        sy[p] = __ffma2_rn(tg, Y2, sy[p]);
        sxy[p] = __ffma2_rn(tg, XY2, sxy[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      S0[2 * p] += s0[p].x;
      S0[2 * p + 1] += s0[p].y;
      SX[2 * p] += sx[p].x;
      SX[2 * p + 1] += sx[p].y;
      SY[2 * p] += sy[p].x;
      SY[2 * p + 1] += sy[p].y;
      SXY[2 * p] += sxy[p].x;
      SXY[2 * p + 1] += sxy[p].y;
      s0[p] = sx[p] = sy[p] = sxy[p] = z2;
    }
    __syncthreads();
  }
  if (ws.evals) {
    for (int off = 16; off > 0; off >>= 1) n_eval += __shfl_xor_sync(0xffffffffu, n_eval, off);
    if ((tid & 31) == 0 && n_eval) atomicAdd(&ws.evals[1], n_eval);
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = ent[k];
    if (e < 0) continue;
    const float4 c = gt[e];
    double *o = gw.entadj + ((size_t)b * max_ent + e) * 3;
    o[0] = S0[k];
    o[1] = SX[k];
    o[2] = (double)c.z * SY[k] + (double)c.w * SXY[k];  // natural-units a_y adjoint
  }
}

// ------------------------------------------------------------------ per-sample chain to theta

typedef Dual<5, double> D5;   // tangents: c0_k, e2_j, s2, c2, b
typedef Dual<9, double> D9;   // tangents: theta 0,1,2,13,14,15,16,17,18
typedef Dual<1, double> DT1;  // one tangent of the delay term (theta 0..7 or H0)


// Table adjoint -> per-Gaussian JAM inputs.  One warp per (tracer k, mass j) pair, lanes
// over the Gauss-Legendre nodes; FP64 duals through the table formula (tangents c0_k, e2_j,
// sin^2 i, cos^2 i, b); warp sums, then one global atomic per quantity and warp.
__global__ void __launch_bounds__(256) k_table_adj(const SysDev *__restrict__ sysv,
                                                   const int *__restrict__ sys_id, WsDev ws,
                                                   GradWs gw, int max_light, int max_mass,
                                                   int max_ent) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 0) return;  // the spherically aligned model has its own adjoint
  const int nMt = S.n_mass_tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kj = blockIdx.x * 8 + warp;
  __shared__ double gsum[8][3];
  double G[7] = {0, 0, 0, 0, 0, 0, 0};  // sum gR, d0 .. d4 (d2..d4 global), unused slot
  const DynP dp = ws.dp[b];
  const size_t bl = (size_t)b * max_light, bm = (size_t)b * max_mass;
  int k = 0, j = 0;
  if (kj < S.n_light * nMt) {
    j = kj % nMt;
    k = kj / nMt;
    const D5 s2 = D5::var(dp.s2, 2), c2 = D5::var(dp.c2, 3), bb = D5::var(dp.b, 4);
    const D5 e2 = D5::var(ws.e2[bm + j], 1);
    const D5 c0 = D5::var(ws.c0[bl + k], 0);
    const double nc = ws.nu0[bl + k] * ws.Cj[bm + j];
    for (int g = lane; g < S.n_gl; g += 32) {
      const int e = kj * S.n_gl + g;
      const double *ga = gw.entadj + ((size_t)b * max_ent + e) * 3;
      const double GQ0 = ga[0], GQ1 = ga[1], Gay = ga[2];
      const double wu = S.gl_wu[e];
      const double a = S.gl_a[e], p = S.gl_p[e];  // u^2/(2 s_j^2), 1/(2 s_k^2) + a
      const D5 h = 1.0 - e2 * S.gl_u2[e];
      const D5 c = c0 + a / h;
      const D5 al = p * s2 + c * c2;
      const D5 sh = dsqrt(h);
      const D5 A = a / (h * sh * c);
      const D5 P0 = A * (bb * s2 + c2);
      const D5 P1 = s2 * (2.0 * a / sh - 2.0 * p * bb * A);
      const D5 wsq = wu * dsqrt(PI_D / al);
      const D5 R0 = wsq * P0, R1 = wsq * P1;
      const D5 ayn = -p * c / al;
      G[0] += GQ0 * R0.v + GQ1 * R1.v;
#pragma unroll
      for (int i = 0; i < 5; ++i) G[1 + i] += nc * (GQ0 * R0.d[i] + GQ1 * R1.d[i]) + Gay * ayn.d[i];
    }
  }
#pragma unroll
  for (int i = 0; i < 6; ++i)
    for (int off = 16; off > 0; off >>= 1) G[i] += __shfl_xor_sync(0xffffffffu, G[i], off);
  double *t = gw.tadj + (size_t)b * gw.tstride;
  const int ML = max_light, MM = max_mass;
  if (lane == 0) {
    if (kj < S.n_light * nMt) {
      // a_nu0[k] += C_j sum gR, a_C[j] += nu0_k sum gR, a_c0[k], a_e2[j]
      atomicAdd(&t[k], ws.Cj[bm + j] * G[0]);
      atomicAdd(&t[ML + k], G[1]);
      atomicAdd(&t[2 * ML + j], ws.nu0[bl + k] * G[0]);
      atomicAdd(&t[2 * ML + MM + j], G[2]);
    }
    gsum[warp][0] = G[3];
    gsum[warp][1] = G[4];
    gsum[warp][2] = G[5];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += gsum[w][threadIdx.x];
    if (v != 0.0) atomicAdd(&t[2 * ML + 2 * MM + threadIdx.x], v);
  }
}

__global__ void __launch_bounds__(256) k_grad_chain(const SysDev *__restrict__ sysv,
                                                    const int *__restrict__ sys_id,
                                                    const double *__restrict__ theta, WsDev ws,
                                                    GradWs gw, int max_light, int max_mass,
                                                    int max_ent, double *grad) {
  const int b = blockIdx.x;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const double *th = theta + (size_t)GLAD_NTHETA * b;
  const int tid = threadIdx.x;
  __shared__ double a_nu0[GLAD_MAX_LIGHT], a_c0[GLAD_MAX_LIGHT];
  __shared__ double a_C[GLAD_MAX_MASS + 1], a_e2[GLAD_MAX_MASS + 1];
  __shared__ double a_glob[4];
  __shared__ double gsm[GLAD_NTHETA];
  __shared__ double Ad[GLAD_MAX_LIGHT][10];  // light amplitudes with tangents (I_e, R_e in slots 3, 4)
  const int nL = S.n_light, nM = S.n_mass, nMt = S.n_mass_tot;
  // (a) the JAM adjoint, carried to nu0_k, c0_k, C_j, e2_j, sin^2 i, cos^2 i, b (and, for the
  // spherically aligned model, the inclination directly) by k_table_adj or k_sph_coef_adj
  {
    const double *t = gw.tadj + (size_t)b * gw.tstride;
    const int ML = max_light, MM = max_mass;
    for (int k = tid; k < nL; k += blockDim.x) {
      a_nu0[k] = t[k];
      a_c0[k] = t[ML + k];
    }
    for (int j = tid; j < nMt; j += blockDim.x) {
      a_C[j] = t[2 * ML + j];
      a_e2[j] = t[2 * ML + MM + j];
    }
    if (tid < 4) a_glob[tid] = t[2 * ML + 2 * MM + tid];
  }
  if (tid < GLAD_NTHETA) gsm[tid] = 0.0;
  __shared__ double sumC;  // sum_j adj(C_j) C_j: the dynamics' derivative by ln(velocity^2 unit)
  if (tid == 0) sumC = 0.0;
  __syncthreads();
  const size_t bl = (size_t)b * max_light;
  // internal mass sheet and distance mode (as in k_prep)
  const double lam = S.sheet ? th[20] : 1.0;
  const double v2u = S.distance_mode == 1 ? S.v2unit * th[22] / th[21] : S.v2unit;
  const int nS = S.n_sheet;

  // (b) per Gaussian: MGE amplitudes (analytic partials of F), deprojection, C_j, e2_j
  const double tE = th[0], g = th[1], q = th[2], inc = th[15];
  const D9 Di = D9::var(inc, 5);
  const D9 si = dsin(Di), ci = dcos(Di);
  const D9 S2 = si * si, C2 = ci * ci;
  const int P2 = 2 * S.mge_P + 1;
  // Euler-inversion sums of each Gaussian and of its partial (R_e for the first lens light,
  // gamma' for the mass), the (Gaussian, node) terms spread over the block
  __shared__ double mf[GLAD_MAX_LIGHT + GLAD_MAX_MASS][2];
  // composite class: light sums are of the Chameleons (f2: d/dw_t of the first), then the
  // halo's (f: of k(u) without kappa_s, f2: of u dk/du), at mf[nL + h]
  const bool comp = S.mass_class == 1;
  const int nE = comp ? nL + S.n_halo : nL + nM;
  for (int k = tid; k < nL + nM; k += blockDim.x) mf[k][0] = mf[k][1] = 0.0;
  __syncthreads();
  {
    const double coef = (3.0 - g) / (1.0 + q) * pow(tE, g - 1.0);
    const double rs2 = S.r_soft * S.r_soft;
    for (int it = tid; it < nE * P2; it += blockDim.x) {
      const int k = it / P2, m = it - k * P2;
      const double2 ch = S.chi[m];
      double f, f2;
      if (comp) {
        if (k < nL) {
          const int cc = S.lcomp_of[k];
          const double qc = S.lcomp[4 * cc + 3];
          const double I0 = cc == 0 ? th[13] : S.lcomp[4 * cc];
          const double wt = cc == 0 ? th[14] : S.lcomp[4 * cc + 2];
          const double A = I0 / (1.0 + qc), sc = 2.0 * S.lcomp[4 * cc + 1] / (1.0 + qc);
          const double st = 2.0 * wt / (1.0 + qc);
          const double sg = S.sig_light[k];
          const cplx z = {sg * ch.x, sg * ch.y};
          const cplx z2 = cmul(z, z);
          const cplx a = cpow_({z2.r + sc * sc, z2.i}, -0.5), bq = cpow_({z2.r + st * st, z2.i}, -0.5);
          f = S.eta[m] * A * (a.r - bq.r);
          const cplx p3 = cpow_({z2.r + st * st, z2.i}, -1.5);
          f2 = cc == 0 ? S.eta[m] * A * st * 2.0 / (1.0 + qc) * p3.r : 0.0;
        } else {
          const double sg = S.sig_mass[k];  // halo Gaussian h = k - nL sits at mass index nL + h = k
          cplx udk;
          const cplx kk = nfw_k_c({sg * ch.x / th[1], sg * ch.y / th[1]}, &udk);
          f = S.eta[m] * kk.r;
          f2 = S.eta[m] * udk.r;
        }
        atomicAdd(&mf[k][0], f);
        atomicAdd(&mf[k][1], f2);
        continue;
      }
      if (k < nL) {
        const int cc = S.lcomp_of[k];
        const double Ie = cc == 0 ? th[13] : S.lcomp[4 * cc];
        const double Re = cc == 0 ? th[14] : S.lcomp[4 * cc + 1];
        const double n = S.lcomp[4 * cc + 2];
        const double bn = sersic_bn_d(n);
        const double sg = S.sig_light[k];
        const cplx z = {sg * ch.x, sg * ch.y};
        const cplx l = clog_({z.r / Re, z.i / Re});
        const cplx w = cexp_({l.r / n, l.i / n});
        const cplx F = cexp_({-bn * (w.r - 1.0), -bn * w.i});
        // dF/dRe = F bn w / (n Re)
        const cplx Fw = cmul(F, w);
        f = S.eta[m] * Ie * F.r;
        f2 = S.eta[m] * Ie * Fw.r * bn / (n * Re);
      } else {
        const double sg = S.sig_mass[k - nL];
        const cplx z = {sg * ch.x, sg * ch.y};
        cplx z2 = cmul(z, z);
        z2.r += rs2;
        const cplx lz = clog_(z2);
        const double ex = -0.5 * (g - 1.0);
        const cplx F = cexp_({ex * lz.r, ex * lz.i});
        // dF/dg = F (-1/(3-g) + ln tE - log(z^2 + rs^2)/2)
        const cplx fac = {-1.0 / (3.0 - g) + log(tE) - 0.5 * lz.r, -0.5 * lz.i};
        const cplx Fg = cmul(F, fac);
        f = S.eta[m] * coef * F.r;
        f2 = S.eta[m] * coef * Fg.r;
      }
      atomicAdd(&mf[k][0], f);
      atomicAdd(&mf[k][1], f2);
    }
  }
  __syncthreads();
  for (int k = tid; k < nL; k += blockDim.x) {
    const int cc = S.lcomp_of[k];
    const double Ie = cc == 0 ? th[13] : S.lcomp[4 * cc];
    const double sg = S.sig_light[k];
    const double f = mf[k][0], fRe = mf[k][1];
    D9 A(S.mw_light[k] * f);
    if (cc == 0) {
      A.d[3] = S.mw_light[k] * f / Ie;
      A.d[4] = S.mw_light[k] * fRe;
    }
    for (int i = 0; i < 10; ++i) Ad[k][i] = i == 0 ? A.v : A.d[i - 1];
    const double qp = S.qp_light[k];
    const D9 qi = dsqrt(qp * qp - C2) / si;
    const D9 nu0 = qp * A / (SQRT2PI_D * sg * qi);
    const D9 c0 = 1.0 / (2.0 * sg * sg * qi * qi);
    const double aI = gw.adjI0[bl + k];
    for (int i = 0; i < 9; ++i) {
      const double v = a_nu0[k] * nu0.d[i] + a_c0[k] * c0.d[i] + aI * A.d[i];
      if (v != 0.0) {
        const int t = i < 3 ? i : (i < 5 ? 10 + i : 10 + i);  // 0,1,2,13,14,15,16,17,18
        atomicAdd(&gsm[t], v);
      }
    }
  }
  __syncthreads();  // Ad (the tracer amplitudes with tangents) complete
  for (int j = tid; j < nM; j += blockDim.x) {
    const double sg = S.sig_mass[j];
    D9 A, qp;
    if (comp && j < nL) {
      // baryons: Upsilon_* L_scale x tracer Gaussian j (tangents I0, w_t of the tracer, Upsilon)
      A.v = Ad[j][0];
      for (int i = 0; i < 9; ++i) A.d[i] = Ad[j][i + 1];
      A = (th[17] * S.L_scale) * A;
      A.d[7] = S.L_scale * Ad[j][0];
      qp = D9(S.qp_light[j]);
    } else if (comp) {
      // halo: kappa_s mw sum eta Re k(u), u = z / r_s; d/d r_s = -kappa_s mw sum eta Re(u k'(u)) / r_s
      const double f = mf[j][0], fu = mf[j][1];
      A = D9(th[0] * S.mw_mass[j] * f);
      A.d[0] = S.mw_mass[j] * f;
      A.d[1] = -th[0] * S.mw_mass[j] * fu / th[1];
      qp = D9::var(q, 2);
    } else {
      const double f = mf[nL + j][0], fg = mf[nL + j][1];
      A = D9(S.mw_mass[j] * f);
      A.d[0] = A.v * (g - 1.0) / tE;
      A.d[1] = S.mw_mass[j] * fg;
      A.d[2] = -A.v / (1.0 + q);
      qp = D9::var(q, 2);
    }
    const D9 qi2 = (qp * qp - C2) / S2;
    const D9 Cj = (2.0 * SQRT2PI_D * v2u * lam * sg) * qp * A;
    const D9 e2 = 1.0 - qi2;
    for (int i = 0; i < 9; ++i) {
      const double v = a_C[j] * Cj.d[i] + a_e2[j] * e2.d[i];
      if (v != 0.0) atomicAdd(&gsm[i < 3 ? i : 10 + i], v);
    }
    const double aC = a_C[j] * Cj.v;
    if (aC != 0.0) {
      if (S.sheet) atomicAdd(&gsm[20], aC / lam);  // C_j proportional to lambda
      atomicAdd(&sumC, aC);
    }
  }
  // the sheet's round Gaussians: C_j = 2 sqrt(2 pi) v2u sigma_j (1 - lambda) A1_j, e2_j = 0
  for (int j = tid; j < nS; j += blockDim.x) {
    const double c1 = 2.0 * SQRT2PI_D * v2u * S.sig_mass[nM + j] * S.sheet_A1[j];
    const double aC = a_C[nM + j];
    if (aC != 0.0) {
      atomicAdd(&gsm[20], -aC * c1);
      atomicAdd(&sumC, aC * c1 * (1.0 - lam));
    }
  }
  __syncthreads();
  __shared__ double sh_mb[10];  // black-hole mass before lambda and its 9 tangents (composite lens)
  if (tid == 0) {
    for (int i = 0; i < 10; ++i) sh_mb[i] = 0.0;
    // black hole: A_BH = f_BH Upsilon L_tot L_scale / (2 pi s^2), L_tot = sum 2 pi A_k s_k^2 q'_k
    if (S.has_bh) {
      D9 L(0.0);
      for (int k = 0; k < nL; ++k) {
        D9 A;
        A.v = Ad[k][0];
        for (int i = 0; i < 9; ++i) A.d[i] = Ad[k][i + 1];
        L = L + (2.0 * PI_D * S.sig_light[k] * S.sig_light[k] * S.qp_light[k]) * A;
      }
      const D9 ups = D9::var(th[17], 7), fbh = D9::var(th[18], 8);
      const double sb = S.bh_sigma;
      const D9 Mb = fbh * ups * L * S.L_scale;
      sh_mb[0] = Mb.v;
      for (int i = 0; i < 9; ++i) sh_mb[1 + i] = Mb.d[i];
      const D9 A = fbh * ups * L * (lam * S.L_scale / (2.0 * PI_D * sb * sb));
      const D9 qi2 = (1.0 - C2) / S2;
      const D9 Cj = 2.0 * SQRT2PI_D * v2u * sb * A;
      const D9 e2 = 1.0 - qi2;
      const int jb = nM + nS;
      for (int i = 0; i < 9; ++i) {
        const double v = a_C[jb] * Cj.d[i] + a_e2[jb] * e2.d[i];
        if (v != 0.0) atomicAdd(&gsm[i < 3 ? i : 10 + i], v);
      }
      const double aC = a_C[jb] * Cj.v;
      if (S.sheet) atomicAdd(&gsm[20], aC / lam);
      atomicAdd(&sumC, aC);
    }
    // globals: sin^2 i, cos^2 i (theta 15) and b = 1/(1-beta) (theta 16)
    gsm[15] += a_glob[0] * S2.d[5] + a_glob[1] * C2.d[5] + a_glob[3];
    const double bb = 1.0 / (1.0 - th[16]);
    gsm[16] += a_glob[2] * bb * bb;
  }
  __syncthreads();
  if (tid >= 32 && tid < 46) {
    // time delays and image positions: -(chi2_tmd + chi2_img)/2 by duals through the FP64
    // lens model, one tangent per thread: theta 0..7, the delay distance (H0 = theta 19 in
    // distance mode 0, D_dt,int = theta 22 in mode 1), lambda_int (theta 20, with a sheet) and,
    // in the composite class, I0, w_t, Upsilon_*, f_BH (theta 13, 14, 17, 18: the baryons and
    // the black hole, whose mass carries its tangent from the chain above)
    const int q = tid - 32;
    const int tmap[14] = {0, 1, 2, 3, 4, 5, 6, 7, S.distance_mode == 1 ? 22 : 19, 20, 13, 14, 17, 18};
    const int t = tmap[q];
    const bool used = q < 9 || (q == 9 && S.sheet) || (q >= 10 && comp);
    if (used) {
      DT1 tt[GLAD_NTHETA];
      for (int i = 0; i < GLAD_NTHETA; ++i) tt[i] = i == t ? DT1::var(th[i], 0) : DT1(th[i]);
      DT1 mbh(sh_mb[0]);
      if (comp && q >= 10) mbh.d[0] = sh_mb[1 + (t == 13 ? 3 : t == 14 ? 4 : t == 17 ? 7 : 8)];
      DT1 chi = chi2_tmd_t<DT1>(tt, S, mbh);
      // image positions: lens parameters (and the sheet) only
      if (S.img_sig && t != 19 && t != 22) chi = chi + chi2_img_t<DT1>(tt, S, mbh);
      atomicAdd(&gsm[t], -0.5 * chi.d[0]);
    }
  }
  __syncthreads();
  if (tid == 0 && S.distance_mode == 1 && sumC != 0.0) {
    // C_j proportional to D_dt,int / D_d
    gsm[22] += sumC / th[22];
    gsm[21] -= sumC / th[21];
  }
  __syncthreads();
  // atomic: the lensing adjoint, on the other stream, may be adding into the same entries
  if (tid < GLAD_NTHETA && gsm[tid] != 0.0) atomicAdd(&grad[(size_t)b * GLAD_NTHETA + tid], gsm[tid]);
}

__global__ void k_grad_zero_invalid(const WsDev ws, int B, double *grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * GLAD_NTHETA) return;
  if (ws.status[i / GLAD_NTHETA] != GLAD_SAMPLE_OK) grad[i] = 0.0;
}

template <class T>
bool galloc(GradWs &w, T *&p, size_t n) {
  void *d = nullptr;
  if (cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return false;
  w.allocs.push_back(d);
  p = (T *)d;
  return true;
}

}  // namespace

void grad_ws_free(glad_ctx *c) {
  if (!c->gws) return;
  for (void *p : c->gws->allocs) cudaFree(p);
  delete c->gws;
  c->gws = nullptr;
}

cudaError_t grad_ws_ensure(glad_ctx *c, int B) {
  if (c->gws && c->gws->B >= B) return cudaSuccess;
  cudaDeviceSynchronize();
  grad_ws_free(c);
  c->gws = new GradWs();
  GradWs &w = *c->gws;
  const size_t b = B;
  const bool ok = galloc(w, w.resid, b * c->max_pix) && galloc(w, w.gpix, b * c->max_pix) &&
                  galloc(w, w.pt, b * c->max_sub) && galloc(w, w.adjpt, 2 * b * c->max_apts) &&
                  galloc(w, w.entadj, b * c->max_ent * 3) && galloc(w, w.adjI0, b * c->max_light);
  w.tstride = 2 * c->max_light + 2 * c->max_mass_tot + 4;
  w.sph_cta = (c->max_sgrid + SPH_GADJ_PTS - 1) / SPH_GADJ_PTS;
  const size_t nc = b * w.sph_cta;
  const bool ok2 = ok && galloc(w, w.tadj, b * w.tstride) && galloc(w, w.sgadj, b * c->max_sgrid) &&
                   galloc(w, w.scoef, nc * c->max_smg * SPH_GADJ_NQ) &&
                   galloc(w, w.strc, nc * c->max_light * 2) && galloc(w, w.sbeta, nc);
  if (!ok2) {
    grad_ws_free(c);
    return cudaErrorMemoryAllocation;
  }
  w.B = B;
  return cudaSuccess;
}

float *grad_resid_buffer(glad_ctx *c) { return c->gws ? c->gws->resid : nullptr; }

cudaError_t launch_jam_fg(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  int tiles = 0;
  for (auto &sd : c->h_sysdev) tiles = std::max(tiles, jam_tiles(sd.nsx, sd.nsy, FG_PTS));
  dim3 grid(tiles, B);
  k_jam_fg<<<grid, JAM_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, *c->gws, c->max_light,
                                         c->max_ent, c->max_bins, c->max_sub);
  return cudaGetLastError();
}

// the accumulators the gradient kernels add into start at zero (before the forward pass)
cudaError_t grad_prepare(glad_ctx *c, int B, double *grad, cudaStream_t st) {
  GradWs &g = *c->gws;
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(double) * GLAD_NTHETA * (size_t)B, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.adjI0, 0, sizeof(double) * c->max_light * (size_t)B, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.tadj, 0, sizeof(double) * g.tstride * (size_t)B, st);
  // tile padding beyond the sky grid must read as g_N = 0
  if (e == cudaSuccess) e = cudaMemsetAsync(g.adjpt, 0, sizeof(float4) * 2 * c->max_apts * (size_t)B, st);
  if (c->n_sph) {
    // samples of the spherically aligned model leave dV/dX, dV/dY at zero for k_kin_adj (their
    // point-coordinate terms come from k_sph_los_adj); their grid adjoint starts at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(g.pt, 0, sizeof(float4) * c->max_sub * (size_t)B, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g.sgadj, 0, sizeof(float2) * c->max_sgrid * (size_t)B, st);
  }
  return e;
}

// lensing adjoint (after k_conv has left the residual weights)
cudaError_t launch_grad_lens(glad_ctx *c, const int *sys_id, int B, double *grad, cudaStream_t st) {
  GradWs &g = *c->gws;
  return GLAD_PROF(c, st, KID_GRAD_LENS, ([&]() -> cudaError_t {
    int max_conv_tiles = 0, max_k = 1;
    for (auto &s : c->sys) {
      const int t = ((s.d.nx + CONV_TX - 1) / CONV_TX) * ((s.d.ny + CONV_TY - 1) / CONV_TY);
      max_conv_tiles = std::max(max_conv_tiles, t);
      max_k = std::max(max_k, s.d.psf_k);
    }
    const int h = (max_k - 1) / 2;
    const size_t smem = sizeof(float) * ((CONV_TX + 2 * h) * (CONV_TY + 2 * h) + max_k * max_k);
    k_conv_adj<<<dim3(max_conv_tiles, B), dim3(CONV_TX, CONV_TY), smem, st>>>(
        c->d_sys, sys_id, c->ws.d, g, c->max_pix);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    bool epl = false, comp = false;
    for (auto &sd : c->h_sysdev) (sd.mass_class == 1 ? comp : epl) = true;
    if (epl)
      k_image_grad<<<dim3(c->max_img_tiles, B), LENS_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, g,
                                                                       c->max_pix, grad);
    if (comp)
      k_image_grad_comp<<<dim3(c->max_img_tiles, B), LENS_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d,
                                                                            g, c->max_pix, grad);
    return cudaGetLastError();
  }()));
}

// dynamics adjoint and the per-sample chain (after k_jam_fg and k_kin_finalize)
cudaError_t launch_grad_dyn(glad_ctx *c, const int *sys_id, const double *theta, int B,
                            double *grad, cudaStream_t st) {
  GradWs &g = *c->gws;
  k_kin_adj<<<dim3(c->max_sky_tiles, B), JAM_THREADS, 0, st>>>(
      c->d_sys, sys_id, c->ws.d, g, c->max_light, c->max_bins, c->max_sub, c->max_apts, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->n_sph) {
    e = GLAD_PROF(c, st, KID_GRAD_SPH, launch_grad_sph(c, sys_id, B, grad, st));
    if (e != cudaSuccess) return e;
  }
  if (c->n_cyl) e = GLAD_PROF(c, st, KID_GRAD_JAM_ADJ, ([&]() -> cudaError_t {
    const int ept = c->tune.adj_ept;
    const int nb = (c->max_ent + ADJ_THREADS * ept - 1) / (ADJ_THREADS * ept);
    if (ept == 2)
      k_jam_adj<2><<<dim3(nb, B), ADJ_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_ent,
                                                        c->max_apts);
    else
      k_jam_adj<4><<<dim3(nb, B), ADJ_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_ent,
                                                        c->max_apts);
    return cudaGetLastError();
  }()));
  if (e != cudaSuccess) return e;
  return GLAD_PROF(c, st, KID_GRAD_CHAIN, ([&]() -> cudaError_t {
    int pairs = 0;
    for (auto &sd : c->h_sysdev) pairs = std::max(pairs, sd.n_light * sd.n_mass_tot);
    if (c->n_cyl) {
      k_table_adj<<<dim3((pairs + 7) / 8, B), 256, 0, st>>>(c->d_sys, sys_id, c->ws.d, g,
                                                           c->max_light, c->max_mass_tot, c->max_ent);
      cudaError_t r0 = cudaGetLastError();
      if (r0 != cudaSuccess) return r0;
    }
    k_grad_chain<<<B, 256, 0, st>>>(c->d_sys, sys_id, theta, c->ws.d, g, c->max_light,
                                    c->max_mass_tot, c->max_ent, grad);
    return cudaGetLastError();
  }()));
}

// zero the gradient of invalid samples (after both branches)
cudaError_t launch_grad_finish(glad_ctx *c, int B, double *grad, cudaStream_t st) {
  k_grad_zero_invalid<<<(B * GLAD_NTHETA + 255) / 256, 256, 0, st>>>(c->ws.d, B, grad);
  return cudaGetLastError();
}

// the entry-parallel adjoint alone, with the context's current shape (for the autotuner)
cudaError_t time_jam_adj(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  GradWs &g = *c->gws;
  const int ept = c->tune.adj_ept;
  const int nb = (c->max_ent + ADJ_THREADS * ept - 1) / (ADJ_THREADS * ept);
  if (ept == 2)
    k_jam_adj<2><<<dim3(nb, B), ADJ_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_ent,
                                                      c->max_apts);
  else
    k_jam_adj<4><<<dim3(nb, B), ADJ_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_ent,
                                                      c->max_apts);
  return cudaGetLastError();
}

void set_grad_smem_limit() {
  const int h = (GLAD_MAX_PSF - 1) / 2;
  const int smem = sizeof(float) * ((CONV_TX + 2 * h) * (CONV_TY + 2 * h) + GLAD_MAX_PSF * GLAD_MAX_PSF);
  cudaFuncSetAttribute(k_conv_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
