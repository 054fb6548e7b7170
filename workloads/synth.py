"""Workload configurations and seeded primitive profiles.

Shapes and profiles follow the Kerr-Schild accretion set-ups of the paper's
results (black hole of mass M and spin a, magnetised gas falling in); the exact
recipes are fixed here so that both sides of every comparison start from the
same numbers:

* noise xi in [-1, 1) from splitmix64(seed, variable, global node index), so it
  does not depend on memory layout, and duplicated interface nodes of adjacent
  radial elements receive the same draw;
* power-law profile: rho_c = 1e-2 r^-1.5;  torus profile:
  rho_c = exp(-((r-10)^2 + (10 cos th)^2)/8) + 1e-4;
* rho = rho_c (1 + 1e-3 xi_rho),  p = 1e-3 rho_c^Gamma (1 + 1e-3 xi_p);
* radial infall v^r = -0.3 sqrt(2M/r) / sqrt(1 + 2M/r)  (contravariant Eulerian
  component; the denominator is a shape factor, not a metric evaluation);
* poloidal field from A_phi = A0 max(rho_c - rho_cut, 0), times sin^2(theta) for the
  theta-independent power-law profiles (regularity on the axis).

Nothing here evaluates the metric or any spectral operator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    M: float = 1.0
    a: float = 0.5
    n_elem: int = 2
    r_min: float = 1.8
    r_max: float = 20.0
    elem_map: int = 1          # 1: log-spaced element bounds, 0: equal widths
    n_r: int = 12
    n_theta: int = 12
    n_phi: int = 16
    # polar band: the BSSN fields of the Kerr-Schild slice are singular on the axis in
    # spherical coordinates, so the grid stops short of the poles
    theta_min: float = math.pi / 8
    theta_max: float = 7 * math.pi / 8
    # 0: Chebyshev-Gauss nodes on [theta_min, theta_max]; 1: the paper's uniform theta grid
    # with a Fourier derivative (whole sphere, theta_min = 0, theta_max = pi)
    theta_basis: int = 0
    gamma_eos: float = 4.0 / 3.0
    profile: str = "powerlaw"  # "powerlaw" | "torus" | "bondi"
    rho0: float = 1e-2         # power-law amplitude
    rho_cut: float = 2e-3      # A_phi threshold
    A0: float = 0.0            # A_phi amplitude
    vphi_amp: float = 0.0      # sub-Keplerian azimuthal velocity amplitude
    noise_amp: float = 1e-3
    seed: int = 1001
    nsteps: int = 1
    cfl: float = 0.3

    @property
    def n_points(self) -> int:
        return self.n_elem * self.n_r * self.n_theta * self.n_phi

    @property
    def shape(self):
        return (self.n_elem, self.n_r, self.n_theta, self.n_phi)


# A0 values put the minimum plasma beta p/(b^2/2) at about 100 (chosen once for each
# profile with the theta band below, and fixed here).
CONFIGS = {
    # one RK3 step, 2 radial elements, 12 x 12 x 16
    "c1": Config("c1", a=0.5, n_elem=2, r_min=1.8, r_max=20.0, n_r=12, n_theta=12,
                 n_phi=16, profile="powerlaw", A0=0.093, seed=1001, nsteps=1),
    # larger single instance: 8 elements, 24 x 32 x 64 (393,216 points), 100 steps
    "c2": Config("c2", a=0.9, n_elem=8, r_min=1.5, r_max=100.0, n_r=24, n_theta=32,
                 n_phi=64, profile="torus", A0=8.4e-3, seed=1002, nsteps=100),
    # precision variant of c1
    "c3": Config("c3", a=0.5, n_elem=2, r_min=1.8, r_max=20.0, n_r=12, n_theta=12,
                 n_phi=16, profile="powerlaw", A0=0.093, seed=1001, nsteps=100),
    # c2's instance on the paper's Fourier theta basis: N_theta = 32 uniform pole-free nodes
    # over the whole sphere (393,216 points), 100 steps
    "c2f": Config("c2f", a=0.9, n_elem=8, r_min=1.5, r_max=100.0, n_r=24, n_theta=32,
                  n_phi=64, theta_min=0.0, theta_max=math.pi, theta_basis=1,
                  profile="torus", A0=8.4e-3, seed=1002, nsteps=100),
    # approximate XCTS initial data (whole sphere, Fourier theta): a dilute power-law gas
    # around the puncture (rho0 = 1e-4: the paper's plain fixed point contracts; at the
    # evolution workloads' densities it diverges); x1 small, x2 on c2f's grid
    "x1": Config("x1", a=0.0, n_elem=2, r_min=1.8, r_max=20.0, n_r=12, n_theta=12, n_phi=16,
                 theta_min=0.0, theta_max=math.pi, theta_basis=1, profile="powerlaw",
                 rho0=1e-4, A0=0.0, seed=1011, nsteps=1),
    "x2": Config("x2", a=0.0, n_elem=8, r_min=1.5, r_max=100.0, n_r=24, n_theta=32, n_phi=64,
                 theta_min=0.0, theta_max=math.pi, theta_basis=1, profile="powerlaw",
                 rho0=1e-4, A0=0.0, seed=1012, nsteps=1),
    # large single instance: 16 elements, 32 x 64 x 128 (4,194,304 points), 200 steps
    "c5": Config("c5", a=0.94, n_elem=16, r_min=1.3, r_max=500.0, n_r=32, n_theta=64,
                 n_phi=128, profile="torus", rho_cut=0.2, A0=8.2e-4, vphi_amp=0.5,
                 seed=1005, nsteps=200),
}


def config(name: str, **overrides) -> Config:
    return dataclasses.replace(CONFIGS[name], **overrides)


def splitmix64(x):
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on uint64 numpy arrays."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def noise(seed: int, var: int, idx):
    """Uniform draw in [-1, 1) keyed on (seed, variable, global node index)."""
    idx = np.asarray(idx, dtype=np.uint64)
    key = np.uint64(((seed & 0xFFFFFF) << 40) ^ ((var & 0x3F) << 34)) ^ idx
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def global_node_index(cfg: Config):
    """Flat index of each node in (E, N_r, N_theta, N_phi), with the two copies of a
    shared radial-element interface node mapped to the same index."""
    E, nr, nt, nph = cfg.shape
    e = np.arange(E).reshape(E, 1, 1, 1)
    i = np.arange(nr).reshape(1, nr, 1, 1)
    k = np.arange(nt).reshape(1, 1, nt, 1)
    l_ = np.arange(nph).reshape(1, 1, 1, nph)
    g = e * (nr - 1) + i
    return ((g * nt + k) * nph + l_).astype(np.uint64)


NOISE_RHO, NOISE_P = 0, 1


def primitive_profiles(cfg: Config, r, theta, phi):
    """Primitive fields on the caller's nodes.

    r, theta, phi: float64 arrays broadcastable to cfg.shape (node coordinates,
    computed by the caller).  Returns a dict of float64 arrays of cfg.shape:
    rho, p, vr, vth, vph (contravariant Eulerian velocity) and A_phi, plus the
    noise-free density rho_c.
    """
    shape = cfg.shape
    r = np.broadcast_to(np.asarray(r, dtype=np.float64), shape)
    th = np.broadcast_to(np.asarray(theta, dtype=np.float64), shape)
    np.broadcast_to(np.asarray(phi, dtype=np.float64), shape)
    M = cfg.M
    if cfg.profile in ("powerlaw", "bondi"):
        rho_c = cfg.rho0 * r ** -1.5
    elif cfg.profile == "torus":
        rho_c = np.exp(-((r - 10.0) ** 2 + (10.0 * np.cos(th)) ** 2) / 8.0) + 1e-4
    else:
        raise ValueError(cfg.profile)
    idx = global_node_index(cfg)
    xr = noise(cfg.seed, NOISE_RHO, idx)
    xp = noise(cfg.seed, NOISE_P, idx)
    rho = rho_c * (1.0 + cfg.noise_amp * xr)
    p = 1e-3 * rho_c ** cfg.gamma_eos * (1.0 + cfg.noise_amp * xp)
    vr = -0.3 * np.sqrt(2.0 * M / r) / np.sqrt(1.0 + 2.0 * M / r)
    vth = np.zeros(shape)
    if cfg.vphi_amp != 0.0:
        vph = cfg.vphi_amp / (r ** 1.5 + cfg.a) * rho_c / rho_c.max()
    else:
        vph = np.zeros(shape)
    A_phi = cfg.A0 * np.maximum(rho_c - cfg.rho_cut, 0.0)
    if cfg.profile in ("powerlaw", "bondi"):
        # a theta-independent A_phi would give B^theta ~ 1/sin(theta) on the axis; the
        # regular form vanishes like sin^2(theta) there
        A_phi = A_phi * np.sin(th) ** 2
    return {"rho": rho, "p": p, "vr": vr, "vth": vth, "vph": vph,
            "A_phi": A_phi, "rho_c": rho_c}


def horizon_radius(M: float, a: float) -> float:
    """Outer horizon radius M + sqrt(M^2 - a^2) (used only to place the inner
    boundary of the batched workload)."""
    return M + math.sqrt(M * M - a * a)


BATCH_BASE_SEED = 1004 * 10 ** 4


def batch_configs(n: int = 256, base_seed: int = BATCH_BASE_SEED):
    """Uneven batch of independent instances: spin a ~ U[0, 0.99], element count
    U{2..8}, order N in {8,12,16,24,32} (N_r = N_theta = N), N_phi in {16,32,64},
    r in [0.9 r_h(a), 50], Bondi-like power-law matter with rho0 ~ U[5e-3, 2e-2]."""
    out = []
    orders = (8, 12, 16, 24, 32)
    nphis = (16, 32, 64)
    for i in range(n):
        s = base_seed + i
        u = [float((splitmix64(np.uint64((s << 8) + j)) >> np.uint64(11))) * 2.0 ** -53
             for j in range(5)]
        a = 0.99 * u[0]
        E = 2 + int(u[1] * 7)
        N = orders[int(u[2] * 5)]
        nph = nphis[int(u[3] * 3)]
        rho0 = 5e-3 + 1.5e-2 * u[4]
        out.append(Config(f"c4_{i}", a=a, n_elem=E, r_min=0.9 * horizon_radius(1.0, a),
                          r_max=50.0, n_r=N, n_theta=N, n_phi=nph, profile="bondi",
                          rho0=rho0, A0=0.05, seed=s, nsteps=10))
    return out
