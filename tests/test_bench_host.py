"""Host logic of bench.py's roofline object (no GPU): the algorithmic work per state, the
FP32-pipe count of the mixed angular kernel, and the choice of the dominant kernel."""
import math

import pytest

import bench
import workloads as W


class _FakeLib:
    """Stands in for the binding's profile-class names."""

    @staticmethod
    def profile_class_names():
        fams = ("radial_synth", "angular", "radial_anal", "dense", "kb")
        return list(fams) + [f + "_f32" for f in fams] + [f + "_df64" for f in fams]


def _profile(entries):
    names = _FakeLib.profile_class_names()
    ms, n = [0.0] * len(names), [0] * len(names)
    for name, (t, k) in entries.items():
        ms[names.index(name)] = t
        n[names.index(name)] = k
    return ms, n


def test_algorithmic_work_per_state_32_atom_cluster():
    """Per-state counts of one H.X on the 32-atom cluster (L = 31, N = 48, 96 x 60 x 120 grid):
    radial 2 N_r N L^2 per direction, Legendre N_theta L^2 N_r per direction (parity folded),
    W V one product per grid point."""
    w = W.erf_cluster_32()
    af = bench.algorithmic_flops(w, 1)
    L, N, nr, nt, nph = 31, 48, 96, 60, 120
    assert af["radial_synth"] == af["radial_anal"] == 2 * nr * N * L * L
    leg = nt * L * L * nr
    assert math.isclose(leg, 5.53e6, rel_tol=1e-3)
    assert af["angular_fp32_pipe"] == 2 * leg + nr * nt * nph
    phi = 2.5 * nph * math.log2(nph) * nr * nt
    assert math.isclose(af["angular"], 2 * leg + 2 * phi + nr * nt * nph)
    assert math.isclose(af["angular"], 35.6e6, rel_tol=2e-3)


def test_roofline_object_is_the_dominant_single_kernel():
    """The aggregate dense class is left out of the choice: with dense largest, the roofline
    object is the mixed angular kernel, rated on its FP32-pipe work against the FP32 peak."""
    pytest.importorskip("torch")
    from paper_1404_3773_gb300 import CS_DF64, CS_MIXED_BF16

    w = W.erf_cluster_32()
    steps = 10
    ms, n = _profile({"dense": (30.7, 180), "angular_f32": (28.2, 160),
                      "angular_df64": (19.1, 10), "radial_synth_f32": (4.3, 160)})
    roof, classes = bench.roofline_table(_FakeLib, w, 46128, 80, CS_MIXED_BF16, ms, n, steps,
                                         CS_DF64)
    assert roof["kernel"] == "angular_f32"
    flops = bench.algorithmic_flops(w, 80)["angular_fp32_pipe"]
    per_ms = 28.2 / 160
    assert roof["flops_per_launch"] == flops
    assert math.isclose(roof["achieved"], flops / (per_ms / 1e3) / 1e12, rel_tol=1e-3)
    assert roof["peak"] == round(bench.FP32_PEAK_TFLOPS, 3)
    assert math.isclose(roof["frac"], roof["achieved"] / roof["peak"], rel_tol=1e-3)
    assert roof["traffic"] == bench.NCU_TRAFFIC_BYTES.get("angular_f32")
    # the FP32 filter's angular class counts all of its work (it runs every stage on FP32)
    from paper_1404_3773_gb300 import CS_FP32
    roof32, _ = bench.roofline_table(_FakeLib, w, 46128, 80, CS_FP32, ms, n, steps, CS_DF64)
    assert roof32["flops_per_launch"] == bench.algorithmic_flops(w, 80)["angular"]
    assert set(classes) == {"dense", "angular_f32", "angular_df64", "radial_synth_f32"}
