"""Host-side pieces of bench.py that feed its roofline object: the algorithmic counts per
launch (the roofline numerator) and the DRAM traffic read from the committed ncu
summaries (a positive figure scaled to the batch while the kernel's sources match the
capture's hash, null otherwise, and null for kernels no summary covers)."""
import bench
from paper_2504_01302_b300 import synth


def test_algorithmic_counts_per_launch():
    systems, B = synth.workload_systems(1)
    sid = [0] * B
    n, _ = bench.sph_exp2_counts(systems, sid, B, "k_jam")
    assert n == B * (60 * 4) ** 2 * 20 * 21 * 32  # sub-samples x tracer x mass(+BH) x u nodes
    systems, B = synth.workload_systems(5)
    n, _ = bench.sph_exp2_counts(systems, sid, B, "k_sph_los")
    assert n == B * (240 * 240) * (32 * 21 + 20)
    n, _ = bench.sph_exp2_counts(systems, sid, B, "k_sph_coef+k_sph_grid")
    assert n == B * 128 * 8 * 65 * (21 * 32 + 20)


def test_traffic_records():
    for kernel, w, grad in (("k_jam", 1, False), ("k_jam_fwd_grad", 1, True),
                            ("k_jam_adjoint", 1, True), ("k_sph_los", 5, False)):
        t64 = bench.ncu_traffic(kernel, w, grad, 64)
        assert t64 is None or (t64 > 0 and bench.ncu_traffic(kernel, w, grad, 128) == 2 * t64), kernel
    assert bench.ncu_traffic("k_sph_adjoint", 5, True, 64) is None
