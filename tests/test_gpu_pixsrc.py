"""Pixelated source reconstruction on the GPU (Sect. 3.1.1, Eqs. s_MP and evi_ext) against the
oracle (oracle/pixsrc.py): the optimal regularisation, the log-evidence there, s_MP, and the
joint logL whose image term the evidence becomes, on the small all-features system with a
square grid and with a ragged one (13 x 11), for the 48^2 and 64^2 systems (PSF sides 7 and
11), in a batch mixed with Sersic-source samples and invalid ones, for a sweep over three grid
resolutions of the same data in one context, and at the RXJ1131-scale workload on a sampled
sample.  Tolerances: ln P and logL 0.05 + 5e-6 |ln P| (the FP32 rays leave ~1e-7 arcsec in
beta, ~1e-6 of a bilinear weight over a source pixel, so a poor fit's data term moves by ~1e-6
of itself, as for the Sersic source, tests/systems.logl_tol), and 0.05 absolute with the rays
in FP64 (precision mode 1); the optimum within 0.05 in ln lambda; s_MP at the GPU's lambda
within 1e-3 of max |s| of the oracle's solution at the same lambda.  Both forms of the evidence
evaluation (one CTA per sample, and the multi-launch form that small batches take by default)
are run on the square, ragged, mixed and RXJ1131-scale cases, and agree with each other."""
import numpy as np
import pytest

from oracle import model, pixsrc
from paper_2504_01302_b300 import synth

from . import systems

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I = synth.IDX


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


def _ctx(sys_list):
    from paper_2504_01302_b300.glad import GladContext
    return GladContext(sys_list)


def pix_system(base, n=(10, 10), half=0.45, th=None):
    th = synth.theta_truth(1) if th is None else th
    c = (th[I["x_src"]], th[I["y_src"]])
    return dict(base, src_pix=1, spx_n=n, spx_box=(c[0] - half, c[0] + half, c[1] - half, c[1] + half))


def oracle_solution_at(th, s, lam):
    grid = pixsrc.grid_of(s)
    m = np.asarray(s["mask"]).ravel() != 0
    from oracle import imaging
    ll = imaging.model_image(th, s, source=False).ravel()
    d = np.asarray(s["data"], np.float64).ravel()[m] - ll[m]
    sig = np.asarray(s["sigma"], np.float64).ravel()[m]
    return pixsrc.solve(pixsrc.response(th, s, grid), d, sig, pixsrc.curvature(grid), lam)


def lnp_tol(ref, rel=5e-6):
    return 0.05 + rel * abs(ref)


def check_against_oracle(ctx, s, th, sys_id=None, b=0, check_s=True, rel=5e-6):
    lam, lnP, sg = ctx.pixsrc(_th(th), sys_id, want_s=True)
    ev = model.evaluate(th[b], s)
    assert ev["status"] == 0
    got_lam, got_lnP = float(lam[b]), float(lnP[b])
    assert abs(got_lnP - ev["lnP"]) < lnp_tol(ev["lnP"], rel), (got_lnP, ev["lnP"])
    assert abs(np.log(got_lam) - np.log(ev["lam"])) < 0.05, (got_lam, ev["lam"])
    if check_s:
        s_ref, _ = oracle_solution_at(th[b], s, got_lam)
        ns = int(np.prod(s["spx_n"]))
        s_gpu = sg.cpu().numpy()[b, :ns]
        assert np.max(np.abs(s_gpu - s_ref)) <= 1e-3 * np.max(np.abs(s_ref)), np.max(np.abs(s_gpu - s_ref))
    return ev


@pytest.fixture(scope="module")
def small():
    s = pix_system(systems.small_system(7))
    return s, _ctx([s])


@pytest.mark.parametrize("path", [1, 2])
def test_square_grid_against_oracle(small, path):
    s, ctx = small
    ctx.set_pix_path(path)
    th = systems.near_truth_thetas(2, seed=201)
    for b in range(2):
        check_against_oracle(ctx, s, th, b=b)
    # the evidence is the image term of logL
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    for b in range(2):
        ev = model.evaluate(th[b], s)
        assert int(st[b]) == 0
        assert abs(float(terms[b, 0]) + 2 * ev["lnP"]) < 2 * lnp_tol(ev["lnP"])
        assert abs(float(logL[b]) - ev["logL"]) < lnp_tol(ev["logL"]), (float(logL[b]), ev["logL"])
    assert ctx.pix_factorizations() > 0
    ctx.set_pix_path(0)


@pytest.mark.parametrize("path", [1, 2])
def test_ragged_grid_and_64px_system(path):
    s = pix_system(systems.small_system(7), n=(13, 11), half=0.5)
    ctx = _ctx([s])
    ctx.set_pix_path(path)
    check_against_oracle(ctx, s, systems.near_truth_thetas(1, seed=203))
    sys_list, ths, _ = model.workload(0)
    s0 = pix_system(sys_list[0], n=(12, 12), half=0.45, th=ths[0])
    ctx = _ctx([s0])
    ctx.set_pix_path(path)
    check_against_oracle(ctx, s0, ths[:1])
    # a poor fit (ln P ~ -8e4): with the rays in FP64 the evidence meets 0.05 absolute
    ctx.set_precision(1)
    check_against_oracle(ctx, s0, ths[:1], rel=0.0)


@pytest.mark.parametrize("path", [1, 2])
def test_mixed_batch_sersic_invalid_and_grid_sweep(path):
    base = systems.small_system(7)
    sweep = [pix_system(base, n=(n, n)) for n in (8, 10, 12)]
    ctx = _ctx([base] + sweep)
    ctx.set_pix_path(path)
    th = systems.near_truth_thetas(6, seed=205)
    th[4, I["q"]] = 1.3  # outside the domain
    sid_np = np.array([0, 1, 2, 3, 2, 0], np.int32)
    sid = torch.as_tensor(sid_np, device="cuda")
    logL, st, terms = ctx.loglike(_th(th), sid, terms=True)
    st = st.cpu().numpy()
    assert st[4] == model.ST_DOMAIN and np.isneginf(float(logL[4]))
    # the Sersic samples are those of a context without the pixelated systems
    ref = _ctx([base]).loglike(_th(th[[0, 5]]))[0].cpu().numpy()
    # same kernels; FP32 shared-memory atomics of the bin sums reorder between launches
    assert np.allclose(logL.cpu().numpy()[[0, 5]], ref, rtol=1e-6, atol=0)
    # every grid of the sweep against the oracle
    for b, si in ((1, 1), (2, 2), (3, 3)):
        check_against_oracle(ctx, sweep[si - 1], th, sid, b=b, check_s=(si == 2))


def test_refusals():
    from paper_2504_01302_b300 import _lib
    s = pix_system(systems.small_system(7))
    ctx = _ctx([s])
    th = _th(systems.near_truth_thetas(1, seed=207))
    with pytest.raises(_lib.GladError):
        ctx.loglike_grad(th)
    with pytest.raises(_lib.GladError):
        ctx.model_image(th[0])


def test_rxj1131_scale_sampled_against_oracle():
    sys_list, th, _ = systems.workload(9)
    s = sys_list[0]
    ctx = _ctx(sys_list)
    B = 16
    out = {}
    for path in (1, 2):
        ctx.set_pix_path(path)
        lam, lnP = ctx.pixsrc(_th(th[:B]))
        logL, st = ctx.loglike(_th(th[:B]))
        assert np.all(st.cpu().numpy() == 0)
        ev = model.evaluate(th[0], s)
        assert abs(float(lnP[0]) - ev["lnP"]) < lnp_tol(ev["lnP"]), (float(lnP[0]), ev["lnP"])
        assert abs(float(logL[0]) - ev["logL"]) < lnp_tol(ev["logL"]), (float(logL[0]), ev["logL"])
        out[path] = (np.log(lam.cpu().numpy()), lnP.cpu().numpy())
    # the two forms: the same arithmetic in another order (the factor's double-float sums,
    # the residual sums' reduction order), so the searches end at the same optimum
    assert np.allclose(out[1][1], out[2][1], rtol=1e-9, atol=1e-3)
    assert np.allclose(out[1][0], out[2][0], rtol=0, atol=1e-3)
    # a batch above 32 samples takes other launch shapes for the trailing tiles (one per CTA):
    # its first 16 samples end where the 16-sample batch did
    ctx.set_pix_path(2)
    lam40, lnP40 = ctx.pixsrc(_th(th[:40]))
    assert np.allclose(lnP40.cpu().numpy()[:B], out[2][1], rtol=1e-9, atol=1e-3)
    assert np.allclose(np.log(lam40.cpu().numpy()[:B]), out[2][0], rtol=0, atol=1e-3)


def test_graph_replay_and_static_refusal(small):
    # the whole search (a fixed number of evaluation passes, converged samples returning at
    # once) is a fixed launch sequence: it captures into a CUDA graph and replays with theta
    # rewritten in place; the allocation-free entry point refuses pixelated-source contexts
    import ctypes as C
    from paper_2504_01302_b300 import _lib
    s, ctx = small
    ta = systems.near_truth_thetas(4, seed=211)
    tb = systems.near_truth_thetas(4, seed=212)
    B = len(ta)
    sid = torch.zeros(B, dtype=torch.int32, device="cuda")
    ref = {k: ctx.loglike(_th(t), sid)[0].cpu().numpy() for k, t in (("a", ta), ("b", tb))}
    theta = _th(ta)
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    status = torch.empty(B, dtype=torch.int32, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = ctx.lib.glad_loglike(ctx.handle, P(sid), P(theta), B, P(logL), P(status), None,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ctx.lib.glad_last_error().decode()
    for k, t in (("a", ta), ("b", tb)):
        theta.copy_(_th(t))
        graph.replay()
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        # shared-memory atomics in the response rows reorder between launches (~1e-7 of F)
        assert np.allclose(logL.cpu().numpy(), ref[k], rtol=1e-6, atol=1e-3)
    rc = ctx.lib.glad_loglike_static(ctx.handle, P(sid), P(theta), B, P(logL), P(status), None, None)
    assert rc == 5 and "pixelated" in ctx.lib.glad_last_error().decode()


@pytest.mark.parametrize("n", [40, 68])
def test_large_grids_against_oracle(n):
    # grids whose response rows need more than the default 48 KB of shared memory (40 x 40)
    # and the largest grid the library takes (68 x 68 = 4,624 pixels, the top of the paper's
    # 60^2 - 68^2 sweep)
    s = pix_system(systems.small_system(7), n=(n, n), half=0.6)
    ctx = _ctx([s])
    th = systems.near_truth_thetas(1, seed=213)
    check_against_oracle(ctx, s, th, check_s=(n == 40))
    if n == 40:
        # one CTA per sample on the same case: the same optimum
        lam2, lnP2 = ctx.pixsrc(_th(th))
        ctx.set_pix_path(1)
        lam1, lnP1 = ctx.pixsrc(_th(th))
        assert abs(float(lnP1[0]) - float(lnP2[0])) < 1e-3 + 1e-9 * abs(float(lnP2[0]))
        assert abs(np.log(float(lam1[0]) / float(lam2[0]))) < 1e-3


def test_composite_class_with_the_dpie_sheet():
    # the pixelated source behind Table 3's joint model: the composite mass class (Chameleons,
    # elliptical NFW halo, black hole) with the internal sheet in distance mode 1
    from .test_gpu_composite import comp_small, near
    s = dict(comp_small(7))
    th = near(2, 215)
    c = (th[0, I["x_src"]], th[0, I["y_src"]])
    # a 12 x 12 grid over +-0.6": lambda ~ 12 at the optimum, F + lambda C conditioned ~2e4.
    # (Over +-0.45" the search ends near lambda ~ 1e-4 with the condition ~3e9: ln P still
    # agrees, being stationary in s, but s_MP then moves by ~1e-3 of max |s| under the FP32
    # Gram entries' ~1e-7 rounding.)
    s.update(src_pix=1, spx_n=(12, 12), spx_box=(c[0] - 0.6, c[0] + 0.6, c[1] - 0.6, c[1] + 0.6))
    ctx = _ctx([s])
    for b in range(2):
        check_against_oracle(ctx, s, th, b=b, check_s=(b == 0))


@pytest.mark.parametrize("iters", [0, 3])
def test_search_ends_early_as_under_capture(iters):
    # eager calls stop enqueueing search passes once no search is open (the host checks a
    # per-pass count); a captured graph records all of them.  Both must give the same optimum
    # and run the same factorisations.  iters 0 is the default cap (40), 3 a cap that ends
    # the searches before they converge.
    import ctypes as C
    s = pix_system(systems.small_system(7), n=(12, 12))
    if iters:
        s = dict(s, spx_iters=iters)
    ctx = _ctx([s])
    th = _th(systems.near_truth_thetas(3, seed=217))
    B = th.shape[0]
    sid = torch.zeros(B, dtype=torch.int32, device="cuda")
    ctx.pix_factorizations()
    lam_e, lnP_e = ctx.pixsrc(th, sid)
    n_e = ctx.pix_factorizations()
    lam = torch.empty(B, dtype=torch.float64, device="cuda")
    lnP = torch.empty(B, dtype=torch.float64, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = ctx.lib.glad_pixsrc(ctx.handle, P(sid), P(th), B, P(lam), P(lnP), None,
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ctx.lib.glad_last_error().decode()
    ctx.pix_factorizations()
    graph.replay()
    torch.cuda.synchronize()
    n_g = ctx.pix_factorizations()
    assert n_e == n_g and n_e >= B
    # the response rows' shared-memory atomics reorder between launches (~1e-7 of F)
    assert np.allclose(lnP.cpu().numpy(), lnP_e.cpu().numpy(), rtol=1e-9, atol=1e-4)
    assert np.allclose(np.log(lam.cpu().numpy()), np.log(lam_e.cpu().numpy()), rtol=0, atol=1e-3)
    if iters:
        assert n_e == iters * B
