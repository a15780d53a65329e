"""Seeded synthetic workloads shared by the GPU path's tests, the oracle's tests
and the benchmark.

This module holds problem sizes, seeds and plain random draws only; none of
the method's arithmetic (no lattice, no KL, no solver, no estimator) lives
here. Seeds are 20180614 + the configuration number.

The five problems follow the paper's experiment setup (Sec. 6: -div(a grad u)=1
on the unit square with zero Dirichlet data, lognormal KL field, FMG per
sample, rank-1 lattice with random shifts), restated on a cell-centred
finite-volume grid with a separable exponential covariance.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20180614


def _cfg(pid, **kw):
    """A problem: id pid (its seed is SEED_BASE + pid) and its parameters."""
    base = dict(
        pid=pid,
        n0=8,
        sigma=1.0,
        corr_len=0.3,
        qoi="mean",
        mu0=2,
        nu1=2,
        nu2=2,
        precision="fp64",
        rtol=0.0,
        max_cycles=60,
        sampler="lattice",
        seed=SEED_BASE + pid,
        R=16,
        log2_nmax=10,
        reuse=True,
    )
    base.update(kw)
    return base


# 1: plain FP64 MG-MLMC with reuse: 4 levels 4x4..32x32, s=10, MC normals,
#    fixed N_l = [512,128,32,8], centre QoI.
MC_4LEVEL = _cfg(1, n_levels=4, n0=4, s=10, qoi="center", sampler="mc", R=1,
                 counts=[512, 128, 32, 8], log2_nmax=32)
# 2: MG-MLQMC in FP64: 6 levels 8x8..256x256, s=100, 2^10 points on level 0
#    halving per level, R=16 shifts, mean-of-u QoI.
LATTICE_6LEVEL = _cfg(2, n_levels=6, s=100, counts=[1024, 512, 256, 128, 64, 32], log2_nmax=10)
# 3: precision form on one finest level of 1024x1024: s=400, lambda=0.1,
#    batches of 256 samples, FP64 refinement to 1e-10 around FP32 cycles.
PRECISION_1024 = _cfg(3, n_levels=8, s=400, corr_len=0.1, precision="mixed_tf32", rtol=1e-10,
                      batch=256, finest=7, log2_nmax=10)
# 4: adaptive MLQMC with reuse, 7 levels 8x8..512x512, s=200, R=16,
#    eps in {1e-2, 3e-3, 1e-3}.
ADAPTIVE_7LEVEL = _cfg(4, n_levels=7, s=200, precision="mixed_tf32", rtol=1e-10,
                       eps=[1e-2, 3e-3, 1e-3], log2_nmax=16)
# 5: large adaptive MLQMC: 9 levels 8x8..2048x2048, s=1000, lambda=0.05, R=16,
#    FMG with fixed mu0 = 2 V(2,2)-cycles per level. One fixed-count step: 16
#    points per shift on the finest level doubling per coarser level
#    (N_l = 4096, 2048, ..., 16 on levels 0..8; 256 finest fields, 130,816
#    samples); adaptive runs to eps = 1e-4.
ADAPTIVE_9LEVEL = _cfg(5, n_levels=9, s=1000, corr_len=0.05, precision="mixed_tf32", rtol=0.0,
                       eps=[1e-4], log2_nmax=12, counts=[16 << (8 - lv) for lv in range(9)])

# 6: multi-index variant, grid level x V-cycle count (one context per cycle
#    count mu0 in {1, 2, 3}): 4 levels 4x4..32x32, s=10, lattice, R=4.
MIMC_4LEVEL = _cfg(6, n_levels=4, n0=4, s=10, R=4, log2_nmax=12, mus=[1, 2, 3], eps=[1e-3])
PROBLEMS = {1: MC_4LEVEL, 2: LATTICE_6LEVEL, 3: PRECISION_1024, 4: ADAPTIVE_7LEVEL, 5: ADAPTIVE_9LEVEL,
            6: MIMC_4LEVEL}


def fixed_count_work(counts, R):
    """Work list for fixed per-level sample counts: one item per level covering
    n = 0..N_l-1 and all R shifts: (level, n_begin, n_end, r_begin, r_end)."""
    return [(lv, 0, int(N), 0, int(R)) for lv, N in enumerate(counts) if N > 0]


def scaled(cfg, **kw):
    """A copy of a configuration with some fields replaced (smaller test cases)."""
    out = dict(cfg)
    out.update(kw)
    return out


def rng(tag: int = 0):
    return np.random.default_rng(SEED_BASE + 1000 + tag)


def random_normals(s, count, tag=0):
    """i.i.d. N(0,1) vectors, shape (count, s)."""
    return rng(tag).standard_normal((count, s))


def random_log_field(n, tag=0, scale=1.0):
    """A rough positive coefficient field exp(scale * N(0,1)) on an n x n grid."""
    return np.exp(scale * rng(tag).standard_normal(n * n))


def random_unit(count, tag=0):
    return rng(tag).random(count)
