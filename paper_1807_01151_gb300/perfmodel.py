"""Algorithmic work model of the eMG kernels (FLOPs and bytes per launch).

Counts what each step of the method must compute in the formulation the kernels use,
independent of how a kernel schedules it.  Used to turn measured kernel times into a
roofline fraction.  Shapes: d dimensions, N modes, q = p + 2 Gauss points per direction,
Q = q^d volume points, QF = q^(d-1) points per face, 2d faces per element, B = 5N.
"""
from dataclasses import dataclass

FMA = 2.0   # FLOPs per fused multiply-add
ROE_FLOPS = 180.0        # one Roe flux evaluation (double), incl. both physical fluxes
FLUX_FLOPS = 30.0        # F_k(U) for all k at one point
FLUXJAC_FLOPS = 40.0     # dF_k/dU for one k at one point


def n_modes(dim, p):
    return (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6


@dataclass
class Shape:
    dim: int
    p: int
    E: int
    F: int          # faces (interior + boundary)

    @property
    def N(self):
        return n_modes(self.dim, self.p)

    @property
    def q(self):
        return self.p + 2

    @property
    def Q(self):
        return self.q ** self.dim

    @property
    def QF(self):
        return self.q ** (self.dim - 1)

    @property
    def B(self):
        return 5 * self.N

    @property
    def NF(self):
        return 2 * self.dim


def residual_face_flops(s):
    """Traces on both sides (2 x 5N FMA) and one Roe flux per face point."""
    return s.F * s.QF * (2 * 5 * s.N * FMA + ROE_FLOPS)


def residual_volume_flops(s):
    """Per element: reconstruction (5N FMA) and flux at Q points, projection on the
    gradients (5N Q d FMA) and on the face traces (5N per face point)."""
    vol = s.Q * (5 * s.N * FMA + FLUX_FLOPS) + 5 * s.N * s.Q * s.dim * FMA if s.p > 0 else 0.0
    return s.E * (vol + s.NF * s.QF * 5 * s.N * FMA)


def residual_bytes(s):
    """State in and residual out (the compulsory traffic; tables are extra)."""
    return 2 * s.E * s.B * 8


def diag_flops(s):
    """Eq. jac1 contraction: per volume point 25 N (d + N) FMA, per face point 25 N (1 + N)."""
    vol = s.Q * (25 * s.N * (s.dim + s.N) * FMA + 5 * s.N * FMA + s.dim * FLUXJAC_FLOPS) if s.p > 0 else 0.0
    face = s.NF * s.QF * 25 * s.N * (1 + s.N) * FMA
    return s.E * (vol + face)


def diag_bytes(s, fb=8):
    """The assembled blocks written once, fb bytes per entry (8: FP64 form, 4: float32 forms)."""
    return s.E * s.B * s.B * fb


def lu_flops(s):
    return s.E * (2.0 / 3.0) * s.B ** 3


def stage_flops(s):
    return s.E * 2.0 * s.B * s.B


def stage_bytes(s, fb=8):
    """Factors (FP64 form) or inverse (float32 forms, fb = 4) read once, residual and u^n in,
    u^(k) out."""
    return s.E * (s.B * s.B * fb + 3 * s.B * 8 + (s.B * 4 if fb == 8 else 0))


def inverse_flops(s):
    """Explicit inverse by Gauss-Jordan (the float32 block forms): 2 B^3 per block."""
    return s.E * 2.0 * s.B ** 3


def vcycle_work(dim, p_max, E, F, rk_stages=4, pre_smooth=2, krylov_m=30, form=0):
    """Per-V-cycle algorithmic FLOPs and compulsory bytes of each kernel class."""
    fb = 8 if form == 0 else 4   # bytes per block entry: FP64 factors or float32 inverses
    w = {k: [0.0, 0.0] for k in ("residual_face_flux", "residual_volume", "diag_block_assembly", "block_lu",
                                 "prk_stage_solve", "arnoldi")}
    # residual evaluations per level: cycle entry (p_max) or forcing (p < p_max),
    # rk_stages - 1 stage residuals per PRK step (+1 for every extra step), 1 for restriction
    for p in range(p_max, -1, -1):
        s = Shape(dim, p, E, F)
        if p == 0:
            n_res = 2      # forcing R_0(v0) and R~_0 for the Krylov start vector
        else:
            n_res = 1 + pre_smooth * rk_stages - 1 + 1
        w["residual_face_flux"][0] += n_res * residual_face_flops(s)
        w["residual_volume"][0] += n_res * residual_volume_flops(s)
        w["residual_face_flux"][1] += n_res * residual_bytes(s) / 2
        w["residual_volume"][1] += n_res * residual_bytes(s) / 2
        if p > 0:
            w["diag_block_assembly"][0] += pre_smooth * diag_flops(s)
            w["diag_block_assembly"][1] += pre_smooth * diag_bytes(s, fb)
            w["block_lu"][0] += pre_smooth * (lu_flops(s) if form == 0 else inverse_flops(s))
            w["block_lu"][1] += pre_smooth * 2 * diag_bytes(s, fb)
            w["prk_stage_solve"][0] += pre_smooth * rk_stages * stage_flops(s)
            w["prk_stage_solve"][1] += pre_smooth * rk_stages * stage_bytes(s, fb)
    K0 = 5 * E
    nf = 2 * dim
    # Arnoldi: m SpMVs over the BSR matrix and CGS2 (two passes of j+1 dots and updates)
    spmv_b = E * (1 + nf) * 25 * 8 + 2 * K0 * 8
    orth_b = sum(2 * 2 * (j + 1) * K0 * 8 for j in range(krylov_m))
    w["arnoldi"][0] = krylov_m * E * (1 + nf) * 25 * FMA + sum(4 * (j + 1) * K0 * FMA for j in range(krylov_m))
    w["arnoldi"][1] = krylov_m * spmv_b + orth_b
    return w
