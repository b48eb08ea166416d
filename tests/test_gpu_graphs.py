"""GMRES restart cycles replayed as CUDA graphs give the same bits as direct
launches, count their kernels, and keep the per-kernel timers working."""
import numpy as np
import pytest
import torch

from paper_1603_04039_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("form", [dict(precision="fp64"), dict(precision="fp64", poly_degree=8, poly_omega=1.0),
                                  dict(precision="mixed", poly_degree=16, poly_omega=1.0)])
def test_graph_replay_is_bit_identical(form):
    """Three ways to run the same solve: direct launches (graphs off) and
    direct launches with kernel timers on, where the host ends a cycle after
    the step whose stopping test passed; graph replays, where the steps after
    that one are skipped on the device (IF nodes).  Same bits and the same
    kernels every way."""
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(60000, 21)
    res = []
    for graphs, timed in ((False, False), (False, True), (True, False)):
        ap = APCloud(max_depth=6, c_refine=0.3, restart=12, **form)
        ap.set_graphs(graphs)
        ap.build_octree(_t(x), _t(y), _t(z))
        ap.stencils()
        ap.deposit(q_uniform=1.0 / len(x), rtol=1e-11)
        if timed:
            ap.set_timing(0xFFFF)
        l0 = ap.launch_count()
        phi, info = ap.solve(rtol=1e-11)
        launches = ap.launch_count() - l0
        ap.set_timing(0)
        php, ex, ey, ez = ap.gather_field()
        st = ap.graph_stats()
        res.append((phi.cpu().numpy(), ex.cpu().numpy(), info["iters"], launches, st))
    for r in res[1:]:
        assert np.array_equal(res[0][0], r[0])
        assert np.array_equal(res[0][1], r[1])
        assert res[0][2] == r[2]
    assert res[0][4]["replays"] == 0 and res[1][4]["replays"] == 0
    assert res[2][4]["replays"] > 0 and res[2][4]["cached"] >= 1
    # a replay counts the kernels that ran: its fixed nodes and the bodies of
    # the steps before the stopping test
    assert res[2][3] == res[1][3] == res[0][3]


def test_timers_inside_graphs():
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(40000, 22)
    out = []
    for graphs in (False, True):
        ap = APCloud(max_depth=6, c_refine=0.4, restart=10)
        ap.set_graphs(graphs)
        ap.build_octree(_t(x), _t(y), _t(z))
        ap.stencils()
        ap.deposit(q_uniform=1.0 / len(x), rtol=1e-11)
        ap.get_timing(reset=True)
        ap.set_timing(0xFFFF)
        ap.solve(rtol=1e-11)
        t = ap.get_timing(reset=True)
        ap.set_timing(0)
        out.append(t)
    for kind in ("spmv", "gmres_dots", "gmres_update_dots", "gmres_update_norm", "gmres_cycle_end"):
        assert out[1][kind][1] == out[0][kind][1], kind     # timed launches
        assert out[1][kind][0] > 0.0, kind                  # milliseconds
        assert out[1][kind][2] == out[0][kind][2], kind     # algorithmic bytes


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_launch_shapes_do_not_change_results(precision):
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(50000, 23)
    res = []
    for bs, ww, un, so in ((256, 4, 1, 0), (64, 2, 4, 1), (512, 8, 1, 1), (128, 4, 4, 0)):
        ap = APCloud(max_depth=6, c_refine=0.3, precision=precision, poly_degree=8, poly_omega=1.0)
        ap.set_launch_shape(bs, ww, un, so)
        ap.build_octree(_t(x), _t(y), _t(z))
        ap.stencils()
        ap.deposit(q_uniform=1.0 / len(x), rtol=1e-11)
        phi, info = ap.solve(rtol=1e-11)
        g = ap.get_stencils()
        res.append((phi.cpu().numpy(), g["D"].cpu().numpy(), g["nbr"].cpu().numpy(), info["iters"]))
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_sweep_l2_keep_does_not_change_results():
    """The sweeps' streaming loads (on every matrix load, on the part past a
    threshold, on none) only steer the caches: the mixed solve gives the same
    bits, replayed from graphs as well as launched directly."""
    from paper_1603_04039_gb300 import APCloud, APCloudError
    x, y, z, q = inputs.beam_with_halo(50000, 25)
    ap = APCloud(max_depth=6, c_refine=0.3, precision="mixed", poly_degree=16, poly_omega=1.0)
    ap.set_launch_shape(128, 4, 4, 1)
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    ap.deposit(q_uniform=1.0 / len(x), rtol=1e-11)
    assert ap.sweep_l2_keep() == 2**63 - 1              # a matrix far below the L2: no streaming loads
    ap.solve(rtol=1e-11)                                 # sets the cycle cap the later solves start from
    res = []
    for graphs in (True, False):
        ap.set_graphs(graphs)
        for keep in (-1, 0, 1 << 20, 1 << 40):
            ap.set_sweep_l2_keep(keep)
            assert ap.sweep_l2_keep() == (2**63 - 1 if keep == -1 else keep)
            phi, info = ap.solve(rtol=1e-11)
            assert info["status"] == 0
            res.append((phi.cpu().numpy(), info["iters"]))
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and r[1] == res[0][1]
    with pytest.raises(APCloudError):
        ap.set_sweep_l2_keep(-2)


@pytest.mark.parametrize("graphs", [True, False])
def test_dependent_launch_does_not_change_results(graphs):
    """Sweeps launched as programmatic dependents of the sweep before them
    give the same bits as sweeps in plain stream order, on the single-system
    and the batched path, replayed from graphs and launched directly."""
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(50000, 26)
    xb, yb, zb, qb, offs, _ = inputs.beam_batch(3, 27, n_lo=5e3, n_hi=2e4)
    res = {}
    for pdl in (False, True):
        ap = APCloud(max_depth=6, c_refine=0.3, precision="mixed", poly_degree=16, poly_omega=1.0)
        ap.set_graphs(graphs)
        ap.set_launch_shape(128, 4, 4, 1)
        ap.set_dependent_launch(pdl)
        # small grids (a few blocks per sweep) let consecutive sweeps share the SMs the most;
        # several solves give an ordering race several chances to show
        runs = []
        for xs, ys, zs, o in ((x, y, z, None), (xb, yb, zb, offs)):
            if o is None:
                ap.build_octree(_t(xs), _t(ys), _t(zs))
            else:
                ap.build_octree_batched(_t(xs), _t(ys), _t(zs), o)
            ap.stencils()
            if o is None:
                ap.deposit(q_uniform=1.0 / len(xs), rtol=1e-11)
            else:
                ap.deposit(q=_t(qb), rtol=1e-11)
            for _ in range(4 if pdl else 1):
                phi, info = ap.solve(rtol=1e-11)
                assert info["status"] == 0
                runs.append((phi.cpu().numpy(), info["iters"]))
        res[pdl] = runs
    ref = res[False]
    for k, (phi, iters) in enumerate(res[True]):
        r_phi, r_iters = ref[k // 4]
        assert np.array_equal(phi, r_phi) and iters == r_iters


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stencil_slots_do_not_change_results(precision):
    """The first stencil pass gathers at most stencil_slots k-ring candidates
    per node; nodes whose rings outgrow them are redone by the second pass with
    512.  With 16 or 32 slots most or many nodes take the second pass: the
    stencils, and the solve, are bit-identical to the default's."""
    from paper_1603_04039_gb300 import APCloud
    x, y, z, q = inputs.beam_with_halo(60000, 28)
    res = []
    for slots in (128, 32, 16):
        ap = APCloud(max_depth=7, c_refine=0.2, precision=precision, poly_degree=8, poly_omega=1.0,
                     stencil_slots=slots)
        ap.build_octree(_t(x), _t(y), _t(z))
        for ww in (4, 8):
            ap.set_launch_shape(256, ww, 1, 0)
            ap.stencils()
        g = ap.get_stencils()
        ap.deposit(q_uniform=1.0 / len(x), rtol=1e-11)
        phi, info = ap.solve(rtol=1e-11)
        res.append([g[k].cpu().numpy() for k in sorted(g)] + [phi.cpu().numpy()])
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_autotune_choices_and_rejects():
    from paper_1603_04039_gb300 import APCloud, APCloudError
    x, y, z, q = inputs.beam_with_halo(80000, 24)
    ap = APCloud(max_depth=6, c_refine=0.3, precision="mixed", poly_degree=16, poly_omega=1.0)
    with pytest.raises(APCloudError) as e:
        ap.autotune()
    assert e.value.status == -7
    ap.build_octree(_t(x), _t(y), _t(z))
    ap.stencils()
    before = ap.get_stencils()["D"].cpu().numpy()
    t = ap.autotune()
    assert t["spmv_block"] in (64, 128, 256, 512) and t["wls_warps"] in (2, 4, 8) and t["spmv_unroll"] in (1, 4)
    assert t["sweep_sorted"] in (0, 1) and len(t["spmv_ms"]) == 16
    assert all(v > 0 for v in t["spmv_ms"].values()) and all(v > 0 for v in t["wls_ms"].values())
    assert np.array_equal(ap.get_stencils()["D"].cpu().numpy(), before)
    _, info = ap.deposit(q_uniform=1.0 / len(x), rtol=1e-10)
    assert info["status"] == 0
    for bad in ((100, 4, 1, 0), (256, 3, 1, 0), (256, 4, 2, 0), (256, 4, 1, 2)):
        with pytest.raises(APCloudError):
            ap.set_launch_shape(*bad)
