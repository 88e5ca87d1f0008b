"""Workload recipes: lattice shapes, operator parameters and seeds.

The paper's measurements use RBC-UKQCD gauge configurations (48^3x96x24 and
32^4, Sec. 6) which are not available here.  Seeded random links
U = exp(i eps H) stand in for them; they are smoother than physical fields
and carry no topology, so iteration counts differ from the paper's.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple          # (Lx, Ly, Lz, Lt)
    Ls: int
    M5: float
    b: float
    c: float
    mass: float
    eps: float
    block: tuple         # fine-block extents
    nvec: int
    tol: float
    prec: str            # fine-operator storage precision
    nrhs: int = 1
    block2: tuple | None = None   # second blocking (on the coarse lattice)
    nvec2: int = 0
    seed: int = 0
    antiperiodic_t: bool = False
    # second-level deflation vectors of the little Dirac operator used by default
    # (0: plain coarse CG).  At m = 0.002 and below, lam_min / lam_max of the
    # coarse operator (~1e-6) is at the level of its FP32 rounding, so the
    # deflation's 1/lam factors are unreliable there; those workloads default to 0.
    ldop_nvec: int = 0
    # set-up of the level-1 subspace: inverse-iteration steps, CG tolerance and
    # iteration cap of each step; and of the level-2 subspace (three levels)
    inv_steps: int = 3
    inv_tol: float = 1e-4
    inv_maxiter: int = 20000
    inv2_steps: int = 2
    inv2_tol: float = 1e-3
    inv2_maxiter: int = 20000
    # order of the Chebyshev polynomial of Q_trunc smoothing the level-1 solve
    # of a three-level workload (0: none; interval from the power iteration)
    qtrunc_order: int = 0
    # storage of the little Dirac operator (None: FP64 for FP64 storage, FP32 for
    # FP32, FP16 for 16-bit); at m = 0.001 an FP16 operator is not positive
    # definite at the bottom of its spectrum, so the three-level workload keeps FP32
    coarse_prec: str | None = None
    extra: dict = field(default_factory=dict)

    @property
    def gauge_seed(self) -> int:
        return 1000 + self.seed

    @property
    def source_seed(self) -> int:
        return 2000 + self.seed

    @property
    def subspace_seed(self) -> int:
        return 3000 + self.seed

    @property
    def coarse_dims(self):
        return tuple(d // bk for d, bk in zip(self.dims, self.block))


WORKLOADS = {
    # plain FP64, tiny; the oracle finishes it in seconds
    "cfg1_8x8x8x8_ls8_shamir": Workload(
        "cfg1_8x8x8x8_ls8_shamir", (8, 8, 8, 8), 8, 1.8, 1.0, 0.0, 0.01, 0.3,
        (4, 4, 4, 4), 8, 1e-10, "f64", seed=1),
    # FP32 fine operator, two-level HDCG
    "cfg2_16x16x16x16_ls16_shamir": Workload(
        "cfg2_16x16x16x16_ls16_shamir", (16, 16, 16, 16), 16, 1.8, 1.0, 0.0, 0.005, 0.35,
        (4, 4, 4, 4), 24, 1e-8, "f32", seed=2, ldop_nvec=64),
    # FP16 storage, Moebius
    "cfg3_24x24x24x48_ls16_mobius": Workload(
        "cfg3_24x24x24x48_ls16_mobius", (24, 24, 24, 48), 16, 1.8, 1.5, 0.5, 0.002, 0.4,
        (4, 4, 4, 4), 32, 1e-8, "f16", seed=3),
    # batched: 12 spin-colour point sources
    "cfg4_24x24x24x48_ls16_mobius_12rhs": Workload(
        "cfg4_24x24x24x48_ls16_mobius_12rhs", (24, 24, 24, 48), 16, 1.8, 1.5, 0.5, 0.002, 0.4,
        (4, 4, 4, 4), 32, 1e-8, "f16", nrhs=12, seed=4),
    # physical-point-like, three levels
    "cfg5_32x32x32x64_ls16_mobius_3lvl": Workload(
        "cfg5_32x32x32x64_ls16_mobius_3lvl", (32, 32, 32, 64), 16, 1.8, 1.5, 0.5, 0.001, 0.45,
        (4, 4, 4, 4), 40, 1e-8, "f16", nrhs=12, block2=(2, 2, 2, 2), nvec2=24, seed=5,
        inv_steps=2, inv_tol=1e-3, inv_maxiter=150, coarse_prec="f32", qtrunc_order=8),
    # Profiling case for the coarse level: the 24^3 x 48 coarse grid and Nvec of
    # cfg3 (an 860 MB FP16 little Dirac operator, larger than L2) over Ls = 2,
    # so the fine subspace stays near 1 GB.
    # Launch-list case of the three-level path: the physical-point-like
    # workload's action, blockings, Nvec and storage on a 16^3 x 32 lattice
    # (1/8 of its volume), so the whole bench run stays within a few minutes.
    "prof_3lvl_16x16x16x32_ls16_mobius": Workload(
        "prof_3lvl_16x16x16x32_ls16_mobius", (16, 16, 16, 32), 16, 1.8, 1.5, 0.5, 0.001, 0.45,
        (4, 4, 4, 4), 40, 1e-8, "f16", nrhs=12, block2=(2, 2, 2, 2), nvec2=24, seed=8,
        inv_steps=2, inv_tol=1e-3, inv_maxiter=150, coarse_prec="f32", qtrunc_order=8),
    # Profiling case for the one-site tensor-core tiles: Nvec 40 (the first
    # level of the three-level workload) on a 4^3 x 8 coarse grid (512 sites;
    # a 531 MB FP32 operator, above L2) over Ls = 2.
    "prof_coarse_16x16x16x32_ls2_nvec40": Workload(
        "prof_coarse_16x16x16x32_ls2_nvec40", (16, 16, 16, 32), 2, 1.8, 1.5, 0.5, 0.001, 0.45,
        (4, 4, 4, 4), 40, 1e-8, "f16", seed=7, coarse_prec="f32"),
    "prof_coarse_24x24x24x48_ls2": Workload(
        "prof_coarse_24x24x24x48_ls2", (24, 24, 24, 48), 2, 1.8, 1.5, 0.5, 0.002, 0.4,
        (4, 4, 4, 4), 32, 1e-8, "f16", seed=6),
}
