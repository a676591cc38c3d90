"""Host logic of bench.py's roofline: the work models of the Krylov kernels
(closed forms over the steps of a solve) and the choice of the roofline kernel."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_krylov_work_closed_forms():
    b = _bench()
    n, nnz, m = 1000, 7000, 50
    for its in (1, 17, 50, 73, 120):
        kw = b.krylov_work(n, nnz, its, m)
        steps = [i % m for i in range(its)]
        sj = sum(steps)
        sjp = sum(max(j - 1, 0) for j in steps)
        assert kw["dgs_next"][0] == 2.0 * (n * sj + its * n)
        assert kw["dgs_spmv_dots"][0] == 2.0 * (n * sj + 2 * n * its + nnz * its)
        assert kw["dgs_fix_adots"][0] == 2.0 * (n * sjp + n * sj + n * its)
        assert kw["dgs_next"][1] == 8 * n * sj + 32 * n * its
    one = b.krylov_work(n, nnz, 0, m, j=25)
    assert one["dgs_next"][0] == 2.0 * (25 * n + n)


def test_roofline_picks_the_largest_modelled_kernel():
    b = _bench()
    n, nnz = 262144, 1810432
    kw = {k: tuple(v) for k, v in b.krylov_work(n, nnz, 42, 50).items()}
    kw["_step"] = {k: tuple(v) for k, v in b.krylov_work(n, nnz, 42, 50, j=25).items()}
    prof = {"dgs_spmv_dots": (3.0, 42), "trsv_up_L0": (3.2, 42), "unmodelled": (9.0, 1), "dgs_next": (1.0, 42)}
    ab = {"trsv_up_L0": 44_000_000}
    rl = b.rooflines(prof, ab, kw, 6800.0, {"hbm_gbs": 6800.0}, "mixed")
    assert [r["kernel"] for r in rl] == ["trsv_up_L0", "dgs_spmv_dots", "dgs_next"]
    assert rl[0]["bound"] == "hbm" and rl[1]["bound"] == "alu"
    t = rl[0]
    assert abs(t["achieved"] - 44e6 / (3.2 / 42 * 1e-3) / 1e9) < 1e-9 and abs(t["frac"] - t["achieved"] / 6800.0) < 1e-12
    k = rl[1]
    assert abs(k["achieved"] - kw["dgs_spmv_dots"][0] / 3.0e-3 / 1e9) < 1e-6
    assert k["peak"] == b.FP64_PEAK_GFLOPS


def test_line_roofline_is_on_the_critical_path():
    """A kernel that runs on the second stream beside M^-1 stays in
    rooflines_top but is not the line's roofline, even with the largest share."""
    b = _bench()
    n, nnz = 262144, 1810432
    kw = {k: tuple(v) for k, v in b.krylov_work(n, nnz, 42, 50).items()}
    kw["_step"] = {k: tuple(v) for k, v in b.krylov_work(n, nnz, 42, 50, j=25).items()}
    prof = {"dgs_fix_adots": (2.8, 42), "trsv_up_L0": (2.7, 42), "dgs_spmv_dots": (2.0, 42)}
    rl = b.rooflines(prof, {"trsv_up_L0": 44_000_000}, kw, 6800.0, {"hbm_gbs": 6800.0}, "mixed")
    assert rl[0]["kernel"] == "dgs_fix_adots"
    assert b.critical_roofline(rl)["kernel"] == "trsv_up_L0"
    only_side = [r for r in rl if r["kernel"] in b.SIDE_STREAM]
    assert b.critical_roofline(only_side)["kernel"] == "dgs_fix_adots"   # nothing else measured


def test_level0_sweep_bytes_of_the_batched_workload():
    """The batched level-0 sweeps' algorithmic bytes, against the figures the
    c4 bench entry reported for the 96-system workload (2,685,836 level-0 rows
    of 2,955,748; 493,891,312 chunk bytes)."""
    b = _bench()
    rows, total, lu = 2_685_836, 2_955_748, 493_891_312
    st = {"lev0_rows": rows, "lev0_l_bytes": lu // 2, "lev0_u_bytes": lu - lu // 2, "lev0_f_nnz": 1000}
    d = b.level0_sweep_bytes(st, total)
    assert d["chunk_bytes"] == lu
    assert d["down_bytes"] == 751_731_568 == lu + 96 * rows
    assert d["up_bytes"] == lu + 8 * 1000 + 8 * rows + 32 * (total - rows) + 96 * rows
