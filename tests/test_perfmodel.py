"""The algorithmic work model behind the roofline fractions (perfmodel.py), checked against
counts made by walking the loops of the contractions and the V-cycle schedule on small shapes
(no GPU)."""
import pytest

from paper_1807_01151_gb300 import perfmodel as pm


def _assembly_fma_by_loops(dim, p, E, nf_faces_per_elem):
    """Eq. jac1 as the assembly evaluates it: at every volume point, for every (a, b, i) the
    contraction over the d gradient directions, then for every (a, b, i, j) the product with
    psi_j; at every face point of every face of the element, psi_i times the face Jacobian
    entry, then the product with psi_j."""
    s = pm.Shape(dim, p, E, 0)
    n = 0
    for _q in range(s.Q if p > 0 else 0):
        for _ab in range(25):
            for _i in range(s.N):
                n += dim                      # sum_k g_k(i) A_k[a][b]
                n += s.N                      # times psi_j, every j
    for _f in range(nf_faces_per_elem):
        for _t in range(s.QF):
            for _ab in range(25):
                for _i in range(s.N):
                    n += 1 + s.N
    return E * n


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1)])
def test_assembly_contraction_count(dim, p):
    s = pm.Shape(dim, p, 3, 0)
    fma = _assembly_fma_by_loops(dim, p, 3, 2 * dim)
    # the model adds, per volume point, the 5N reconstruction FMAs and d flux Jacobians
    extra = 3 * (s.Q * (5 * s.N * pm.FMA + dim * pm.FLUXJAC_FLOPS) if p > 0 else 0.0)
    assert pm.diag_flops(s) == pytest.approx(fma * pm.FMA + extra, rel=1e-15)


def test_stage_bytes_count_the_stored_precision():
    """FP64 form: the LU factors (8 bytes per entry) and the pivot indices; float32 forms: the
    explicit inverse at 4 bytes per entry; both read r and u^n and write u^(k) in FP64."""
    s = pm.Shape(2, 4, 10, 0)
    B = 75
    assert pm.stage_bytes(s) == 10 * (B * B * 8 + 3 * B * 8 + B * 4)
    assert pm.stage_bytes(s, 4) == 10 * (B * B * 4 + 3 * B * 8)
    assert pm.diag_bytes(s, 4) * 2 == pm.diag_bytes(s)


def _residuals_per_cycle(p_max, pre_smooth, rk_stages):
    """Residual evaluations of one V-cycle (Sec. 2.3), walked step by step: R at the cycle
    entry on p_max; on every level the PRK steps (the first stage of the first step reuses the
    entry or forcing residual, every other stage evaluates one); after smoothing R_p(v) for the
    restriction and R_{p-1}(v0) for the forcing; on p = 0 the forcing and the EXP1 right-hand
    side."""
    per_level = {p: 0 for p in range(p_max + 1)}
    per_level[p_max] += 1                       # cycle entry (norm and first stage)
    for p in range(p_max, 0, -1):
        for step in range(pre_smooth):
            for k in range(1, rk_stages + 1):
                if step == 0 and k == 1:
                    continue                    # R~_p(u^n) already available
                per_level[p] += 1
        per_level[p] += 1                       # R~_p(v_p) for the restriction
        per_level[p - 1] += 1                   # R_{p-1}(v0_{p-1}) for tau_{p-1}
    per_level[0] += 1                           # R~_0 for the EXP1 step
    return per_level


@pytest.mark.parametrize("p_max", [1, 2, 4])
def test_residual_count_per_cycle(p_max):
    counts = _residuals_per_cycle(p_max, 2, 4)
    w = pm.vcycle_work(2, p_max, 7, 13, rk_stages=4, pre_smooth=2)
    expect = sum(n * pm.residual_volume_flops(pm.Shape(2, p, 7, 13)) for p, n in counts.items())
    assert w["residual_volume"][0] == pytest.approx(expect, rel=1e-15)
    # 128x64 cylinder at p = 4: 38 evaluations per cycle (the bench's launch count per class)
    if p_max == 4:
        assert sum(counts.values()) == 38


def test_kernel_rooflines_divide_model_work_by_measured_time():
    """bench.py's per-class rooflines: ALU classes report FLOPs / time against the pipe's peak
    (FP64 for the FP64 form's block kernels, FP32 for the float32 forms), HBM classes bytes /
    time against the copy bandwidth."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    work = pm.vcycle_work(2, 4, 8192, 16512, form=1)
    prof = {k: {"ms_per_cycle": 2.0} for k in work}
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 80.0}
    out = bench.kernel_rooflines(prof, work, peaks, 6800.0, 1)
    for k, v in out.items():
        if v["bound"] == "alu":
            assert v["achieved"] == pytest.approx(work[k][0] / 2e-3 / 1e12)
        else:
            assert v["achieved"] == pytest.approx(work[k][1] / 2e-3 / 1e9)
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
    assert out["block_lu"]["peak"] == 80.0 and out["residual_volume"]["peak"] == 1.0
    assert out["prk_stage_solve"]["bound"] == "hbm" and out["prk_stage_solve"]["peak"] == 6800.0
    assert bench.kernel_rooflines(prof, pm.vcycle_work(2, 4, 8192, 16512, form=0), peaks, 6800.0,
                                  0)["block_lu"]["peak"] == 1.0
