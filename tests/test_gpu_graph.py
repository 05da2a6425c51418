"""Uneven batching under a CUDA graph: the 8 uneven systems (64..256 px, ss 1-3, 8-30
Gaussians per component, 20-120 bins, GL 24-64) and 1024 samples split over them, with the
persistent work-list form of the JAM pair sum pinned, captured once into a CUDA graph
(glad_loglike at B = 1024, glad_loglike_grad at B = 64) and replayed twice with theta
rewritten in place between the replays.  Each replay must reproduce the eager call on the
same theta (same kernels: only the order of FP64 atomic sums may differ) and, on sampled
samples of the cheaper systems, the oracle (tolerances of test_gpu_parity)."""
import numpy as np
import pytest

from oracle import model
from paper_2504_01302_b300 import synth

from . import systems
from .test_gpu_grad import assert_grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PERSISTENT = 100000 + 8042  # 8 points per thread, 4 CTAs/SM, unroll 2, persistent form
# replay against eager call: the same kernels, but FP32 atomic sums (bin accumulators in shared
# memory) and FP64 atomics reorder between runs, ~1e-7 relative in each chi^2 term
SAME = 1e-6


@pytest.fixture(scope="module")
def uneven():
    from paper_2504_01302_b300.glad import GladContext
    sys_list = systems.uneven_systems()
    th, sid = synth.workload_thetas(3, 1024, len(sys_list))
    rng = np.random.Generator(np.random.PCG64(3201))
    th2 = synth.draw_prior(rng, 1024)
    ctx = GladContext(sys_list)
    ctx.set_tuning(PERSISTENT, 4)
    return sys_list, th, th2, sid, ctx


def _near(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    fin = np.isfinite(a)
    assert np.array_equal(fin, np.isfinite(b))
    scale = np.abs(a[fin]) if a.ndim == 1 else np.max(np.abs(a[fin]))
    assert np.all(np.abs(a[fin] - b[fin]) <= rel * scale + 1e-9), np.max(np.abs(a[fin] - b[fin]))


def test_graph_replay_matches_eager_and_oracle(uneven):
    import ctypes as C
    sys_list, th_a, th_b, sid_np, ctx = uneven
    B = len(th_a)
    theta = torch.as_tensor(th_a, device="cuda")
    sid = torch.as_tensor(sid_np, device="cuda")
    # eager references (these calls also size the workspace: nothing is allocated in capture)
    ref = {}
    for name, t in (("a", th_a), ("b", th_b)):
        l, st, terms = ctx.loglike(torch.as_tensor(t, device="cuda"), sid, terms=True)
        ref[name] = (l.cpu().numpy(), st.cpu().numpy(), terms.cpu().numpy())
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    status = torch.empty(B, dtype=torch.int32, device="cuda")
    terms = torch.empty(B, 4, dtype=torch.float64, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = ctx.lib.glad_loglike(ctx.handle, P(sid), P(theta), B, P(logL), P(status), P(terms),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ctx.lib.glad_last_error().decode()
    for name, t in (("a", th_a), ("b", th_b)):
        theta.copy_(torch.as_tensor(t, device="cuda"))  # theta changed in place, graph unchanged
        logL.fill_(0.0)
        graph.replay()
        torch.cuda.synchronize()
        l_ref, st_ref, terms_ref = ref[name]
        assert np.array_equal(status.cpu().numpy(), st_ref)
        assert int((st_ref == 0).sum()) > B // 4
        _near(l_ref, logL.cpu().numpy(), SAME)
        ok = st_ref == 0
        # each chi^2 term within SAME of the sample's total chi^2
        tr, tg = terms_ref[ok], terms.cpu().numpy()[ok]
        tot = np.sum(np.abs(tr), axis=1, keepdims=True)
        assert np.all(np.abs(tr - tg) <= SAME * tot + 1e-9)
    # sampled samples of the replayed batch (theta b) against the oracle: the first valid
    # sample of each of the two cheapest systems (fewest sky sub-samples x table entries)
    cost = [(s["kx"] * s["kss"]) * (s["ky"] * s["kss"]) * sum(s["n_mge_light"]) *
            (s["n_mge_mass"] + 1) * s["n_gl"] for s in sys_list]
    got = logL.cpu().numpy()
    st = status.cpu().numpy()
    for si in np.argsort(cost)[:2]:
        b = int(next(i for i in np.flatnonzero(sid_np == si) if st[i] == 0))
        ev = model.evaluate(th_b[b], sys_list[si])
        assert ev["status"] == 0
        assert abs(got[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (si, b, got[b], ev["logL"])


def test_graph_replay_of_the_gradient(uneven):
    import ctypes as C
    sys_list, th_a, th_b, sid_np, ctx = uneven
    B = 64
    # near-posterior draws over all eight systems, two parameter sets
    ta = systems.near_truth_thetas(B, seed=3301)
    tb = systems.near_truth_thetas(B, seed=3302)
    sid_np = (np.arange(B) % len(sys_list)).astype(np.int32)
    sid = torch.as_tensor(sid_np, device="cuda")
    ref = {}
    for name, t in (("a", ta), ("b", tb)):
        l, g, st = ctx.loglike_grad(torch.as_tensor(t, device="cuda"), sid)
        ref[name] = (l.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy())
    theta = torch.as_tensor(ta, device="cuda")
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty(B, synth.N_THETA, dtype=torch.float64, device="cuda")
    status = torch.empty(B, dtype=torch.int32, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = ctx.lib.glad_loglike_grad(ctx.handle, P(sid), P(theta), B, P(logL), P(grad), P(status),
                                       None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ctx.lib.glad_last_error().decode()
    for name, t in (("a", ta), ("b", tb)):
        theta.copy_(torch.as_tensor(t, device="cuda"))
        grad.fill_(0.0)
        graph.replay()
        torch.cuda.synchronize()
        l_ref, g_ref, st_ref = ref[name]
        assert np.array_equal(status.cpu().numpy(), st_ref) and np.all(st_ref == 0)
        _near(l_ref, logL.cpu().numpy(), SAME)
        g = grad.cpu().numpy()
        # FP64 atomics reorder between calls: bound at the gradient scale of each sample
        for b in range(B):
            assert np.all(np.abs(g[b] - g_ref[b]) <= 1e-6 * np.abs(g_ref[b]) +
                          1e-7 * np.max(np.abs(g_ref[b]))), b
    # one replayed sample of the cheapest system against oracle differences, every component
    cost = [(s["kx"] * s["kss"]) * (s["ky"] * s["kss"]) * sum(s["n_mge_light"]) *
            (s["n_mge_mass"] + 1) * s["n_gl"] for s in sys_list]
    si = int(np.argmin(cost))
    b = int(np.flatnonzero(sid_np == si)[0])
    assert_grad_close(grad.cpu().numpy()[b], systems.oracle_grad_fd_pool(tb[b], sys_list[si]))
