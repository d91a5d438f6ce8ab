"""Seeded synthetic inputs and the named workload configurations.

This module holds no arithmetic of the method: it only draws reproducible
inputs (weights, spin configurations, time series) that both the CUDA path
and the CPU oracle consume, and names the workload sizes.

Workloads (the paper's temperatures, Sec. I: T1 = 2.0 second order, T2 = 1.0
and T3 = 0.9 first order, Tt = 1.4182 near the tricritical point):
  small     L=8,  T=2.0,    64 walkers,   10 iterations x 200 sweeps, seed 0
  medium    L=16, T=1.0,    1024 walkers, 30 iterations x 500 sweeps, seed 1
  mixed     L in {8,12,16,20,24,32} x T in {2.0,1.4182,1.0,0.9}, 512 walkers
            each, 20 iterations x 300 sweeps in one CUDA graph, seed 2
  large     L=48, T=0.9,    4096 walkers, 40 x 1000 sweeps + 10^4 measurement
            sweeps, seed 3
  reweight  4096 walkers x 10^4 samples of (E_J, E_Delta, M) shaped like an
            L=32, T=1.4182 multicanonical run, reweighted to a 4096-point Delta
            grid spanning +-0.05 around the transition
"""
import numpy as np

TEMPS = (2.0, 1.4182, 1.0, 0.9)

SMALL = dict(L=8, T=2.0, n_walkers=64, n_iter=10, sweeps=200, seed=0)
MEDIUM = dict(L=16, T=1.0, n_walkers=1024, n_iter=30, sweeps=500, seed=1)
MIXED = dict(Ls=(8, 12, 16, 20, 24, 32), Ts=TEMPS, n_walkers=512, n_iter=20, sweeps=300, seed=2)
LARGE = dict(L=48, T=0.9, n_walkers=4096, n_iter=40, sweeps=1000, n_meas=10000, seed=3)
# The disordered model: bimodal couplings j1, j2 (ratio 0.6, mean 4) on every
# bond with probability 1/2 each, at T = 3.6 (T = 0.9 in units of the mean
# coupling); 4096 walkers of L = 24, one realisation.
DISORDERED = dict(L=24, T=3.6, n_walkers=4096, j1=5, j2=3, bond_seed=11, sweeps=100, seed=6)
REWEIGHT = dict(L=32, T=1.4182, n_walkers=4096, n_samples=10000, n_grid=4096, half_width=0.05,
                seed=4)


def mixed_groups(n_walkers=MIXED["n_walkers"], Ls=MIXED["Ls"], Ts=MIXED["Ts"]):
    return [{"L": L, "T": T, "n_walkers": n_walkers} for L in Ls for T in Ts]


def random_lnW(n_e, seed, scale=1.0, slope=0.0):
    """A rough random weight function (a random walk plus a linear slope)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, scale, n_e)) + slope * np.arange(n_e)


def random_spins(n_walkers, V, seed, values=(-1, 0, 1)):
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(values, dtype=np.int8), size=(n_walkers, V))


def synthetic_series(L=REWEIGHT["L"], T=REWEIGHT["T"], n_walkers=REWEIGHT["n_walkers"],
                     n_samples=REWEIGHT["n_samples"], seed=REWEIGHT["seed"], delta_t=2.8446):
    """A synthetic multicanonical time series of an L^3 lattice.

    E_Delta is spread flat over [0, V] (what a converged multicanonical run
    samples); the weights lnW(E) are chosen so that the reweighted E_Delta
    distribution has two peaks of equal height at Delta = delta_t (a
    spin-0-rich phase near e = 0.25 and a spin-(+-1)-rich phase near e = 0.8),
    with smooth per-walker correlations in time.  E_J and M are drawn around
    E_Delta-dependent means.  Returns (e_j, e_d, m) int32 arrays shaped
    [n_samples][n_walkers], lnW [V + 1] and delta_t."""
    rng = np.random.default_rng(seed)
    V = L ** 3
    beta = 1.0 / T
    E = np.arange(V + 1, dtype=np.float64)
    e = E / V
    # a double-well log density of states at Delta = delta_t, barrier height
    # growing like L^2 (an interface), peaks of equal height
    well = -((e - 0.25) * (e - 0.8)) ** 2 / 0.01
    log_g = beta * delta_t * E + (0.6 * L * L) * (well - well.max())
    lnW = -log_g
    # per-walker random walk in E_Delta, reflected into [0, V]
    step = max(1, V // 200)
    x = rng.integers(0, V + 1, n_walkers).astype(np.int64)
    ed = np.empty((n_samples, n_walkers), dtype=np.int64)
    for s in range(n_samples):
        x = x + rng.integers(-step, step + 1, n_walkers)
        x = np.where(x < 0, -x, x)
        x = np.where(x > V, 2 * V - x, x)
        ed[s] = x
    ef = ed / V
    ej = -3.0 * V * ef ** 2 * (0.4 + 0.6 * ef) + rng.normal(0.0, np.sqrt(V), ed.shape)
    mag = V * ef * np.clip((ef - 0.4) / 0.4, 0.0, 1.0) + rng.normal(0.0, np.sqrt(V), ed.shape)
    sign = np.where(rng.random(n_walkers) < 0.5, -1.0, 1.0)
    m = np.clip(np.rint(mag * sign), -ed, ed)
    return (np.rint(ej).astype(np.int32), ed.astype(np.int32), m.astype(np.int32), lnW,
            delta_t)


def random_bonds(L, j1, j2, seed, p2=0.5):
    """A quenched bimodal bond realisation: int8 [L^3][3], the forward x, y,
    z bond of every site independently j2 with probability p2, else j1
    (integer couplings; the random-bond model with ratio r = j2 / j1)."""
    rng = np.random.default_rng(seed)
    pick = rng.random((L ** 3, 3)) < p2
    return np.where(pick, j2, j1).astype(np.int8)


def delta_grid(center, half_width=REWEIGHT["half_width"], n=REWEIGHT["n_grid"]):
    return center - half_width + (2.0 * half_width) * np.arange(n) / (n - 1)
