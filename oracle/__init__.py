"""FP64 CPU oracle for the periodic single-hop energy change and the KMC step.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package, and this package
never imports the product.  Both sides share only the seeded input generators
in ``workloads``, which hold none of the method's arithmetic.

Definition followed (Sec. 2.2.1 periodic images, Sec. 2.2.2 / App. B boundary
at infinity, Sec. 3.1 periodic near/far split of the hop energy): the tinfoil
Ewald energy of a neutral cubic cell,

    U  = 1/2 sum_i sum_j sum'_n q_i q_j / |r_i - r_j + n a|,
    dU = q_k [phi_{-k}(r') - phi_{-k}(r)],  phi_{-k}(x) = sum_{j != k} q_j psi(x - r_j).

The Ewald pair potential psi and everything that is O(N) per proposal live in
plain C (``kmc_oracle.c``).  The lattice site potential for large grids is a
circular convolution of the charge grid with the tabulated psi, done with a
library FFT (numpy) as one step.

Parity status: psi, psi_reg(0), the energy, dU and the KMC selection are
pinned by tests against the NaCl Madelung constant, brute-force cubic-shell
image sums with Richardson extrapolation, beta independence, hop reversal,
lattice symmetries, U(after) - U(before) and a chi-square test of selection
frequencies.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

DEFAULT_BETA_A = 4.5  # beta * a; with one real-space image shell erfc(1.5*4.5) ~ 1e-21


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP).  Returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I64, I, P = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        sig = {
            "oracle_default_kmax": (I, [D]),
            "oracle_num_threads": (I, []),
            "oracle_psi": (D, [D, D, I, I, D, D, D]),
            "oracle_psi_reg0": (D, [D, D, I, I]),
            "oracle_energy": (D, [I64, P, P, D, D, I, I]),
            "oracle_delta_u": (D, [I64, P, P, D, D, I, I, I64, P]),
            "oracle_delta_u_many": (None, [I64, P, P, D, D, I, I, I64, P, P, P]),
            "oracle_psi_table": (None, [I64, D, I, I, P]),
            "oracle_site_potential": (None, [I64, P, I64, P, P, P]),
            "oracle_site_update": (None, [I64, P, P, I64, I64, D]),
            "oracle_hop_target": (I64, [I64, I64, I]),
            "oracle_hop_targets": (None, [I64, I64, P, I, P]),
            "oracle_hop_vector": (None, [I, P]),
            "oracle_lattice_delta_u": (None, [I64, P, P, I64, P, P, P, P, P]),
            "oracle_lattice_delta_u_list": (None, [I64, P, P, P, P, I64, P, P, P]),
            "oracle_lattice_delta_u_direct": (None, [I64, P, I64, P, P, I64, P, P, P]),
            "oracle_rates": (None, [I64, P, P, D, P]),
            "oracle_select": (I64, [I64, P, D, D, P, P]),
            "oracle_cumsum": (None, [I64, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def ewald_params(a: float, beta_a: float = DEFAULT_BETA_A):
    """(beta, kmax) for box edge a."""
    lib = _load()
    return beta_a / a, int(lib.oracle_default_kmax(beta_a))


# ---------------------------------------------------------------- pair potential
def psi(a: float, d, beta_a: float = DEFAULT_BETA_A, nreal: int = 1, kmax: int | None = None) -> float:
    """Tinfoil Ewald pair potential psi(d) for a cubic box of edge a."""
    lib = _load()
    beta, k = ewald_params(a, beta_a)
    if kmax is not None:
        k = kmax
    return float(lib.oracle_psi(a, beta, nreal, k, float(d[0]), float(d[1]), float(d[2])))


def psi_reg0(a: float, beta_a: float = DEFAULT_BETA_A, nreal: int = 1, kmax: int | None = None) -> float:
    """lim_{d->0} psi(d) - 1/|d| (self-image potential)."""
    lib = _load()
    beta, k = ewald_params(a, beta_a)
    if kmax is not None:
        k = kmax
    return float(lib.oracle_psi_reg0(a, beta, nreal, k))


def energy(pos: np.ndarray, q: np.ndarray, a: float, beta_a: float = DEFAULT_BETA_A) -> float:
    """Total tinfoil energy U (O(N^2) pair potentials; small systems only)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    beta, k = ewald_params(a, beta_a)
    return float(lib.oracle_energy(len(q), _p(pos), _p(q), a, beta, 1, k))


def delta_u(pos: np.ndarray, q: np.ndarray, a: float, particle, target,
            beta_a: float = DEFAULT_BETA_A) -> np.ndarray:
    """dU for each (particle[t], target[t]) proposal, direct O(N) Ewald sum each."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    particle = np.ascontiguousarray(np.atleast_1d(particle), dtype=np.int64)
    target = np.ascontiguousarray(np.asarray(target, dtype=np.float64).reshape(-1, 3))
    out = np.empty(len(particle), dtype=np.float64)
    beta, k = ewald_params(a, beta_a)
    lib.oracle_delta_u_many(len(q), _p(pos), _p(q), a, beta, 1, k, len(particle), _p(particle),
                            _p(target), _p(out))
    return out


# ---------------------------------------------------------------- lattice mode
_table_cache: dict = {}


def psi_table(E: int, beta_a: float = DEFAULT_BETA_A) -> np.ndarray:
    """G[d] = psi(d) on the E^3 integer displacement grid (spacing 1), G[0] = psi_reg(0).

    Flat array indexed d = dx + E*(dy + E*dz)."""
    key = (int(E), float(beta_a))
    if key in _table_cache:
        return _table_cache[key]
    lib = _load()
    beta, k = ewald_params(float(E), beta_a)
    G = np.empty(E ** 3, dtype=np.float64)
    lib.oracle_psi_table(E, beta, 1, k, _p(G))
    _table_cache[key] = G
    return G


def site_potential(E: int, G: np.ndarray, sites: np.ndarray, q: np.ndarray, method: str = "auto") -> np.ndarray:
    """phi_s = sum_j q_j G[s - s_j] for all E^3 sites (includes the j = s self term G[0])."""
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if method == "auto":
        method = "direct" if E ** 3 * len(q) <= 2e9 else "fft"
    if method == "direct":
        lib = _load()
        phi = np.empty(E ** 3, dtype=np.float64)
        lib.oracle_site_potential(E, _p(G), len(q), _p(sites), _p(q), _p(phi))
        return phi
    # circular convolution of the charge grid with G, via a library FFT
    rho = np.zeros(E ** 3, dtype=np.float64)
    np.add.at(rho, sites, q)
    rho = rho.reshape(E, E, E)
    g = G.reshape(E, E, E)
    phi = np.fft.irfftn(np.fft.rfftn(rho) * np.fft.rfftn(g), s=(E, E, E), axes=(0, 1, 2))
    return np.ascontiguousarray(phi.reshape(-1))


def lattice_delta_u_direct(E: int, G: np.ndarray, sites, q, particle, target_site) -> np.ndarray:
    """dU by the direct O(N) sum over the other charges (tabulated psi), per proposal."""
    lib = _load()
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    particle = np.ascontiguousarray(particle, dtype=np.int64)
    target_site = np.ascontiguousarray(target_site, dtype=np.int64)
    out = np.empty(len(particle), dtype=np.float64)
    lib.oracle_lattice_delta_u_direct(E, _p(G), len(q), _p(sites), _p(q), len(particle), _p(particle),
                                      _p(target_site), _p(out))
    return out


def hop_target(E: int, s: int, k: int) -> int:
    return int(_load().oracle_hop_target(E, s, k))


def hop_vectors(nhop: int = 6) -> np.ndarray:
    """The oracle's hop set (Algorithm 5; Sec. 5.3 for 14 hops): nhop x 3 integer lattice offsets,
    the faces (+x, -x, +y, -y, +z, -z), then the body diagonals with x varying fastest."""
    if nhop not in (6, 14):
        raise ValueError("hop sets have 6 or 14 hops")
    lib = _load()
    out = np.empty((nhop, 3), dtype=np.int64)
    for k in range(nhop):
        lib.oracle_hop_vector(k, _p(out[k]))
    return out


def hop_targets(E: int, sites, nhop: int = 6) -> np.ndarray:
    """Target site of every hop of every charge, (n, nhop), event order j = nhop i + k, periodic."""
    if nhop not in (6, 14):
        raise ValueError("hop sets have 6 or 14 hops")
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), nhop), dtype=np.int64)
    _load().oracle_hop_targets(int(E), len(sites), _p(sites), int(nhop), _p(out))
    return out


class LatticeState:
    """Lattice KMC state in the oracle: sites, charges, occupancy and the site potential.

    Hop directions k = 0..5 are (+x, -x, +y, -y, +z, -z); event index j = 6 i + k."""

    def __init__(self, E: int, sites: np.ndarray, q: np.ndarray, beta_a: float = DEFAULT_BETA_A,
                 method: str = "auto"):
        self.E = int(E)
        self.sites = np.array(sites, dtype=np.int64)
        self.q = np.array(q, dtype=np.float64)
        self.n = len(self.q)
        self.G = psi_table(self.E, beta_a)
        self.occ = np.zeros(self.E ** 3, dtype=np.uint8)
        self.occ[self.sites] = 1
        self.phi = site_potential(self.E, self.G, self.sites, self.q, method)

    def propose(self):
        lib = _load()
        dU = np.empty(6 * self.n, dtype=np.float64)
        mask = np.empty(6 * self.n, dtype=np.uint8)
        lib.oracle_lattice_delta_u(self.E, _p(self.G), _p(self.phi), self.n, _p(self.sites), _p(self.q),
                                   _p(self.occ), _p(dU), _p(mask))
        return dU.reshape(self.n, 6), mask.reshape(self.n, 6)

    def delta_u_list(self, particle, target_site) -> np.ndarray:
        lib = _load()
        particle = np.ascontiguousarray(particle, dtype=np.int64)
        target_site = np.ascontiguousarray(target_site, dtype=np.int64)
        out = np.empty(len(particle), dtype=np.float64)
        lib.oracle_lattice_delta_u_list(self.E, _p(self.G), _p(self.phi), _p(self.sites), _p(self.q),
                                        len(particle), _p(particle), _p(target_site), _p(out))
        return out

    def energy(self) -> float:
        """U = 1/2 sum_i q_i phi_{s_i} (phi includes the self-image term q_i G[0])."""
        return float(0.5 * np.dot(self.q, self.phi[self.sites]))

    def target(self, i: int, k: int) -> int:
        return hop_target(self.E, int(self.sites[i]), int(k))

    def accept(self, i: int, k: int) -> None:
        self.accept_site(i, self.target(i, k))

    def accept_site(self, i: int, s_new: int) -> None:
        """Move charge i to lattice site s_new (any hop set) and update the site potential."""
        s_old = int(self.sites[i])
        s_new = int(s_new)
        if self.occ[s_new]:
            raise ValueError("target site occupied")
        lib = _load()
        lib.oracle_site_update(self.E, _p(self.G), _p(self.phi), s_old, s_new, float(self.q[i]))
        self.occ[s_old] = 0
        self.occ[s_new] = 1
        self.sites[i] = s_new


# ---------------------------------------------------------------- KMC step
def rates(dU: np.ndarray, mask: np.ndarray | None, kT: float) -> np.ndarray:
    lib = _load()
    dU = np.ascontiguousarray(dU, dtype=np.float64).reshape(-1)
    out = np.empty_like(dU)
    if mask is None:
        lib.oracle_rates(len(dU), _p(dU), None, kT, _p(out))
    else:
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        lib.oracle_rates(len(dU), _p(dU), _p(mask), kT, _p(out))
    return out


def select(rate: np.ndarray, zeta: float, xi: float):
    """(j, Q, dt): j with R_{j-1} < Q zeta <= R_j, sequential FP64 cumulative sum."""
    lib = _load()
    rate = np.ascontiguousarray(rate, dtype=np.float64).reshape(-1)
    Q = ctypes.c_double()
    dt = ctypes.c_double()
    j = lib.oracle_select(len(rate), _p(rate), zeta, xi, ctypes.byref(Q), ctypes.byref(dt))
    return int(j), float(Q.value), float(dt.value)


def cumsum(rate: np.ndarray) -> np.ndarray:
    lib = _load()
    rate = np.ascontiguousarray(rate, dtype=np.float64).reshape(-1)
    out = np.empty_like(rate)
    lib.oracle_cumsum(len(rate), _p(rate), _p(out))
    return out


def kmc_step(state: LatticeState, kT: float, zeta: float, xi: float):
    """One rejection-free KMC step on the lattice state; returns (j, dt, Q, dU, mask)."""
    dU, mask = state.propose()
    r = rates(dU, mask, kT)
    j, Q, dt = select(r, zeta, xi)
    if j >= 0:
        state.accept(j // 6, j % 6)
    return j, dt, Q, dU, mask


# ---------------------------------------------------------------- free space
# Free-space boundary conditions (Sec. 2.2 before the periodic case; Sec. 3,
# Eq. (proposed_energy)): a finite charge distribution in unbounded space, no
# images and no neutrality condition.  The definitions, summed directly in
# FP64 (numpy), are
#   U  = 1/2 sum_{i != j} q_i q_j / |r_i - r_j|,
#   dU = q_k sum_{j != k} q_j (1/|r' - r_j| - 1/|r_k - r_j|)   (charge k: r_k -> r').
# Parity status: pinned by closed forms (two charges, a square of alternating
# charges), U(after) - U(before), hop reversal and rigid-motion invariance.

def free_energy(pos: np.ndarray, q: np.ndarray) -> float:
    """Free-space energy, direct pair sum (each pair once)."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    U = 0.0
    for i in range(len(q) - 1):
        r = np.sqrt(np.sum((pos[i + 1:] - pos[i]) ** 2, axis=1))
        U += q[i] * np.sum(q[i + 1:] / r)
    return float(U)


def free_delta_u(pos: np.ndarray, q: np.ndarray, particle, target, chunk: int = 512) -> np.ndarray:
    """Free-space dU of moving charge particle[t] to target[t]; NaN where the
    target coincides with another charge or with the charge itself."""
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    particle = np.atleast_1d(np.asarray(particle, dtype=np.int64))
    target = np.asarray(target, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(particle), dtype=np.float64)
    chunk = max(1, min(chunk, 4_000_000 // max(len(q), 1)))  # bounded temporaries
    for c0 in range(0, len(particle), chunk):
        pk = particle[c0:c0 + chunk]
        tk = target[c0:c0 + chunk]
        d_new = np.sqrt(np.sum((tk[:, None, :] - pos[None, :, :]) ** 2, axis=2))
        d_old = np.sqrt(np.sum((pos[pk][:, None, :] - pos[None, :, :]) ** 2, axis=2))
        rows = np.arange(len(pk))
        with np.errstate(divide="ignore", invalid="ignore"):
            inv_new = 1.0 / d_new
            inv_old = 1.0 / d_old
        inv_new[rows, pk] = 0.0  # the moving charge itself
        inv_old[rows, pk] = 0.0
        v = q[pk] * ((inv_new - inv_old) @ q)
        singular = np.any(d_new == 0.0, axis=1) | np.all(tk == pos[pk], axis=1)
        v[singular] = np.nan
        out[c0:c0 + chunk] = v
    return out


# ---------------------------------------------------------------- Dirichlet walls
# Grounded walls (phi = 0) at z = 0 and z = a/2 with an applied field E_z along
# z, periodic in x and y (Sec. 2.2, Dirichlet, Fig. dirichlet_bc_domain): the
# physical charges sit on lattice sites with z index < E/2; each has a mirror
# of opposite charge at z index E - 1 - z (position a - z); the mirrored cell
# of edge a is replicated periodically (tinfoil).  Then
#   U_phys = 1/2 U_ext - E_z sum_i q_i z_i,
# and a hop moves the charge and its mirror together:
#   dU_phys = 1/2 [U_ext(after) - U_ext(before)] - q E_z dz.
# With psi the periodic pair potential, dU_1 = q[phi_{-i}(r') - phi_{-i}(r)]
# the single-charge change in the mirrored system and m the mirror, the mirror
# symmetry of the other charges gives
#   dU_phys = dU_1 - q^2/2 [psi(r' - r'_m) - 2 psi(r' - r_m) + psi(r - r_m)] - q E_z dz.
# Parity status: pinned by the vanishing potential on both walls and by the
# brute-force Ewald energies of the mirrored system before and after a move.

def mirror_sites(E: int, sites: np.ndarray) -> np.ndarray:
    """Site of each charge's mirror image: (x, y, z) -> (x, y, E - 1 - z)."""
    xyz = np.stack([sites % E, (sites // E) % E, sites // (E * E)], axis=1)
    return xyz[:, 0] + E * (xyz[:, 1] + E * (E - 1 - xyz[:, 2]))


class DirichletLattice:
    """Lattice KMC state between grounded walls (see above); event j = nh i + k over the
    physical charges, hops from ``hop_vectors`` (integer lattice offsets, (nh, 3))."""

    def __init__(self, E: int, sites: np.ndarray, q: np.ndarray, hop_vectors: np.ndarray, field_z: float = 0.0,
                 beta_a: float = DEFAULT_BETA_A):
        self.E, self.n, self.field_z = int(E), len(q), float(field_z)
        sites = np.asarray(sites, dtype=np.int64)
        if np.any(sites // (E * E) >= E // 2):
            raise ValueError("physical charges must sit below the mirror plane z = a/2")
        self.hops = np.asarray(hop_vectors, dtype=np.int64)
        q = np.asarray(q, dtype=np.float64)
        self.ext = LatticeState(E, np.concatenate([sites, mirror_sites(E, sites)]), np.concatenate([q, -q]), beta_a)

    @property
    def sites(self) -> np.ndarray:
        return self.ext.sites[: self.n]

    def _G(self, dxyz: np.ndarray) -> np.ndarray:
        E = self.E
        d = np.mod(dxyz, E)
        return self.ext.G[d[..., 0] + E * (d[..., 1] + E * d[..., 2])]

    def energy(self) -> float:
        q = self.ext.q[: self.n]
        z = (self.sites // (self.E * self.E)) + 0.5
        return 0.5 * self.ext.energy() - self.field_z * float(np.dot(q, z))

    def propose(self):
        """(dU[n, nh], mask[n, nh]); masked: the target is occupied or beyond a wall."""
        E, n, nh = self.E, self.n, len(self.hops)
        s = self.sites
        xyz = np.stack([s % E, (s // E) % E, s // (E * E)], axis=1)
        raw = xyz[:, None, :] + self.hops[None, :, :]
        t = np.mod(raw, E)
        ts = t[..., 0] + E * (t[..., 1] + E * t[..., 2])
        inside = (raw[..., 2] >= 0) & (raw[..., 2] < E // 2)
        mask = inside & (self.ext.occ[ts] == 0)
        dU = np.full((n, nh), np.nan)
        ii, kk = np.nonzero(mask)
        d1 = self.ext.delta_u_list(ii, ts[ii, kk])
        q = self.ext.q[ii]
        z, zn = xyz[ii, 2], raw[ii, kk, 2]
        h = self.hops[kk]
        zero = np.zeros_like(z)
        g_new_mir = self._G(np.stack([zero, zero, 2 * zn + 1 - E], axis=1))   # r' - r'_m
        g_cross = self._G(np.stack([h[:, 0], h[:, 1], z + zn + 1 - E], axis=1))  # r' - r_m
        g_old_mir = self._G(np.stack([zero, zero, 2 * z + 1 - E], axis=1))    # r - r_m
        dU[ii, kk] = d1 - 0.5 * q * q * (g_new_mir - 2.0 * g_cross + g_old_mir) - q * self.field_z * (zn - z)
        return dU, mask.astype(np.uint8)

    def accept(self, i: int, target_site: int) -> None:
        self.ext.accept_site(i, int(target_site))
        self.ext.accept_site(i + self.n, int(mirror_sites(self.E, np.array([target_site]))[0]))
