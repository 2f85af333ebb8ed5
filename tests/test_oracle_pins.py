"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, a wrong image or index) fails at least one of them:

* Madelung constant of rock salt (closed value, golden file) -- pins psi,
  psi_reg(0) and the lattice table / FFT site potential together.
* beta independence of psi -- pins the relative weight of real and
  reciprocal parts and the -pi/(beta^2 V) constant.
* brute-force cubic-shell image sums with Richardson extrapolation on tiny
  boxes -- pins the tinfoil reading of the boundary at infinity (Sec. 2.2.2,
  App. B): U_cubic = U_tinfoil + 2 pi |M|^2 / (3V).
* hop reversal, lattice translation, 90-degree rotation and charge
  conjugation invariances of dU; direct (off-lattice) dU equal to the lattice
  table dU; U(after) - U(before) = dU.
* the KMC selection rule (Algorithm 1) against an independent numpy version,
  and a chi-square test of event frequencies.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out[parts[0]] = float(parts[1])
    return out


# ----------------------------------------------------------------- psi itself
@pytest.mark.parametrize("E", [2, 4, 8])
def test_madelung_rock_salt(E):
    M = _golden("madelung.txt")["nacl"]
    s = np.arange(E ** 3)
    xyz = workloads.site_xyz(E, s)
    q = (-1.0) ** xyz.sum(1)
    G = oracle.psi_table(E)
    for method in ("direct", "fft"):
        phi = oracle.site_potential(E, G, s, q, method=method)
        U = 0.5 * np.dot(q, phi[s])
        assert abs(U / E ** 3 + M / 2) < 1e-12, (method, U / E ** 3)


def test_madelung_direct_energy():
    """The O(N^2) off-lattice energy path reproduces the same constant."""
    M = _golden("madelung.txt")["nacl"]
    E = 4
    s = np.arange(E ** 3)
    pos = workloads.site_positions(E, s)
    q = (-1.0) ** workloads.site_xyz(E, s).sum(1)
    U = oracle.energy(pos, q, float(E))
    assert abs(U / E ** 3 + M / 2) < 1e-12


@pytest.mark.parametrize("d", [(1.5, 0.5, 0.5), (7.5, 3.0, 2.0), (0.3, 0.2, 0.1), (8.0, 8.0, 8.0),
                               (-3.25, 11.0, 0.0)])
def test_psi_beta_independent(d):
    a = 16.0
    ref = oracle.psi(a, d)
    scale = max(abs(ref), 1.0 / a)
    for ba, nreal, kmax in ((3.5, 2, 8), (5.5, 2, 12), (6.5, 2, 14)):
        v = oracle.psi(a, d, beta_a=ba, nreal=nreal, kmax=kmax)
        assert abs(v - ref) < 1e-13 * scale, (ba, v, ref)


def test_psi_reg0_beta_independent():
    a = 10.0
    ref = oracle.psi_reg0(a)
    for ba, nreal, kmax in ((3.5, 2, 8), (5.5, 2, 12)):
        assert abs(oracle.psi_reg0(a, beta_a=ba, nreal=nreal, kmax=kmax) - ref) < 1e-13


def test_psi_singular_limit():
    """psi(d) - 1/|d| -> psi_reg(0) as d -> 0 (the regular part is smooth, so
    the gap shrinks like |d|^2)."""
    a = 8.0
    p0 = oracle.psi_reg0(a)
    gaps = []
    for eps in (1e-1, 5e-2):
        d = np.array([0.6, -0.3, 0.74]) * eps
        gaps.append(abs(oracle.psi(a, d) - 1.0 / np.linalg.norm(d) - p0))
    assert gaps[1] < gaps[0] / 3.0 and gaps[1] < 1e-3


def test_psi_periodic_and_even():
    a = 6.0
    d = np.array([1.3, -2.2, 0.4])
    v = oracle.psi(a, d)
    assert abs(oracle.psi(a, d + a * np.array([1, -2, 3])) - v) < 1e-13
    assert abs(oracle.psi(a, -d) - v) < 1e-13


def test_table_matches_pointwise_psi():
    E = 8
    G = oracle.psi_table(E)
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.integers(0, E, size=3)
        if not d.any():
            continue
        idx = d[0] + E * (d[1] + E * d[2])
        assert abs(G[idx] - oracle.psi(float(E), d.astype(float))) < 1e-13
    assert abs(G[0] - oracle.psi_reg0(float(E))) < 1e-14


# ------------------------------------------------- boundary at infinity (tinfoil)
def _cubic_shell_energy(pos, q, a, K):
    """U_K = 1/2 sum_ij sum_{|n|_inf <= K}' q_i q_j / |r_i - r_j + n a|, and the
    energy of the last shell (for the trapezoid end correction)."""
    n = len(q)
    U = 0.0
    for i in range(n):
        for j in range(n):
            if i != j:
                U += 0.5 * q[i] * q[j] / np.linalg.norm(pos[i] - pos[j])
    last = 0.0
    for k in range(1, K + 1):
        r = np.arange(-k, k + 1)
        nn = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
        nn = nn[np.abs(nn).max(1) == k]
        d = pos[:, None, None, :] - pos[None, :, None, :] + a * nn[None, None, :, :]
        last = 0.5 * np.einsum("i,j,ijn->", q, q, 1.0 / np.linalg.norm(d, axis=-1))
        U += last
    return U, last


def _extrapolated_cubic_energy(pos, q, a, K=24):
    """Richardson extrapolation of the cubic-shell sum (end-corrected so that
    the remainder is c/K^2 + O(K^-4))."""
    UK, lastK = _cubic_shell_energy(pos, q, a, K)
    UH, lastH = _cubic_shell_energy(pos, q, a, K // 2)
    tK = UK - 0.5 * lastK
    tH = UH - 0.5 * lastH
    return (4.0 * tK - tH) / 3.0


@pytest.mark.parametrize("seed", [5, 11])
def test_tinfoil_equals_cubic_sum_minus_surface_term(seed):
    rng = np.random.default_rng(seed)
    a = 4.0
    n = 6
    pos = rng.random((n, 3)) * a
    q = np.array([1.0, -1.0, 1.0, -1.0, 2.0, -2.0])
    U_cubic = _extrapolated_cubic_energy(pos, q, a)
    M = (q[:, None] * pos).sum(0)
    surf = 2.0 * np.pi / (3.0 * a ** 3) * float(M @ M)
    U_t = oracle.energy(pos, q, a)
    assert abs(U_t + surf - U_cubic) < 2e-7
    # the surface term is not negligible here, so a sign error would be seen
    assert surf > 1e-3


def test_hop_energy_against_brute_force():
    """dU of one hop from the oracle equals the brute-force cubic-shell energy
    difference after removing the change of the surface term."""
    rng = np.random.default_rng(21)
    a = 4.0
    pos = rng.random((4, 3)) * a
    q = np.array([1.0, -1.0, 1.0, -1.0])
    tgt = np.array([0.3, 3.7, 1.1])
    new = pos.copy()
    new[2] = tgt

    def tinfoil_from_cubic(p):
        M = (q[:, None] * p).sum(0)
        return _extrapolated_cubic_energy(p, q, a) - 2.0 * np.pi / (3.0 * a ** 3) * float(M @ M)

    dU_bf = tinfoil_from_cubic(new) - tinfoil_from_cubic(pos)
    dU = oracle.delta_u(pos, q, a, [2], [tgt])[0]
    assert abs(dU - dU_bf) < 4e-7


def test_near_image_constant():
    """The paper's printed self-image constant (Sec. 3.1): sum over the 26
    nearest images of 1/|nu| = 6 + 8/sqrt(3) + 12/sqrt(2) ~ 19.104."""
    g = _golden("paper_constants.txt")["near_image_inverse_distance_sum"]
    r = np.arange(-1, 2)
    nu = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    nu = nu[np.abs(nu).sum(1) > 0]
    s = float(np.sum(1.0 / np.linalg.norm(nu, axis=1)))
    assert abs(s - (6 + 8 / math.sqrt(3) + 12 / math.sqrt(2))) < 1e-12
    assert abs(s - g) < 5e-4


# ------------------------------------------------------------ dU invariants
def _state(E=8, N=40, seed=7):
    sites, q = workloads.random_small(E, N, seed)
    return oracle.LatticeState(E, sites, q)


def test_hop_then_reverse_sums_to_zero():
    st = _state()
    dU, mask = st.propose()
    rev = {0: 1, 1: 0, 2: 3, 3: 2, 4: 5, 5: 4}
    checked = 0
    for i in range(0, st.n, 3):
        for k in range(6):
            if not mask[i, k]:
                continue
            d1 = dU[i, k]
            st2 = oracle.LatticeState(st.E, st.sites, st.q)
            st2.accept(i, k)
            d2, m2 = st2.propose()
            assert m2[i, rev[k]]
            assert abs(d1 + d2[i, rev[k]]) < 1e-12 * max(1.0, abs(d1))
            checked += 1
            break
    assert checked > 5


def test_translation_invariance():
    E = 8
    st = _state(E)
    dU, mask = st.propose()
    xyz = workloads.site_xyz(E, st.sites)
    for shift in ((1, 0, 0), (0, 3, 0), (2, 5, 7)):
        t = (xyz + np.array(shift)) % E
        s2 = t[:, 0] + E * (t[:, 1] + E * t[:, 2])
        st2 = oracle.LatticeState(E, s2, st.q)
        d2, m2 = st2.propose()
        assert np.array_equal(mask, m2)
        assert np.nanmax(np.abs(d2 - dU)) < 1e-12


def test_rotation_invariance():
    """90 degrees about z: (x, y) -> (E-1-y, x); hops +x->+y, -x->-y, +y->-x, -y->+x."""
    E = 8
    st = _state(E)
    dU, mask = st.propose()
    xyz = workloads.site_xyz(E, st.sites)
    t = np.stack([E - 1 - xyz[:, 1], xyz[:, 0], xyz[:, 2]], 1)
    s2 = t[:, 0] + E * (t[:, 1] + E * t[:, 2])
    st2 = oracle.LatticeState(E, s2, st.q)
    d2, m2 = st2.propose()
    perm = [2, 3, 1, 0, 4, 5]  # new direction of old hop k
    for k in range(6):
        assert np.array_equal(mask[:, k], m2[:, perm[k]])
        ok = mask[:, k] == 1
        assert np.max(np.abs(dU[ok, k] - d2[ok, perm[k]])) < 1e-12


def test_charge_conjugation_invariance():
    st = _state()
    dU, mask = st.propose()
    st2 = oracle.LatticeState(st.E, st.sites, -st.q)
    d2, m2 = st2.propose()
    assert np.nanmax(np.abs(dU - d2)) < 1e-12


def test_direct_equals_table():
    """Off-lattice direct Ewald dU agrees with the lattice table dU."""
    E = 8
    st = _state(E, N=24, seed=9)
    dU, mask = st.propose()
    pos = workloads.site_positions(E, st.sites)
    parts, tgts, ref = [], [], []
    for i in range(st.n):
        for k in range(6):
            if mask[i, k]:
                parts.append(i)
                tgts.append(workloads.site_positions(E, [st.target(i, k)])[0])
                ref.append(dU[i, k])
    d = oracle.delta_u(pos, st.q, float(E), parts, tgts)
    assert np.max(np.abs(d - np.array(ref))) < 1e-12


def test_lattice_direct_sum_equals_site_potential_form():
    """The O(N)-per-hop direct sum and the maintained site potential agree."""
    E = 8
    st = _state(E, N=60, seed=37)
    dU, mask = st.propose()
    parts, tg, ref = [], [], []
    for i in range(st.n):
        for k in range(6):
            if mask[i, k]:
                parts.append(i)
                tg.append(st.target(i, k))
                ref.append(dU[i, k])
    d = oracle.lattice_delta_u_direct(E, st.G, st.sites, st.q, parts, tg)
    assert np.max(np.abs(d - np.array(ref))) < 1e-12


def test_energy_difference_equals_delta_u():
    E = 6
    sites, q = workloads.random_small(E, 10, 13)
    st = oracle.LatticeState(E, sites, q)
    pos = workloads.site_positions(E, sites)
    U0 = oracle.energy(pos, q, float(E))
    assert abs(U0 - st.energy()) < 1e-12
    dU, mask = st.propose()
    i, k = [(i, k) for i in range(st.n) for k in range(6) if mask[i, k]][3]
    st.accept(i, k)
    U1 = oracle.energy(workloads.site_positions(E, st.sites), q, float(E))
    assert abs((U1 - U0) - dU[i, k]) < 1e-12
    assert abs(st.energy() - U1) < 1e-12


def test_fft_site_potential_equals_direct():
    E = 16
    sites, q = workloads.random_small(E, 200, 17)
    G = oracle.psi_table(E)
    a = oracle.site_potential(E, G, sites, q, method="direct")
    b = oracle.site_potential(E, G, sites, q, method="fft")
    assert np.max(np.abs(a - b)) < 1e-12


def test_hop_sets_are_the_lattice_neighbour_shells():
    """The oracle's hop sets against a brute-force enumeration of the lattice neighbours
    (Algorithm 5; Sec. 5.3 for 14 hops): 6 faces at distance 1 in the order +x, -x, +y, -y,
    +z, -z, then the 8 body diagonals at distance sqrt(3) with x varying fastest and + before
    -; the targets are those offsets wrapped periodically."""
    cube = [(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)]
    faces = [v for v in cube if sum(c * c for c in v) == 1]
    diag = [v for v in cube if sum(c * c for c in v) == 3]
    v6, v14 = oracle.hop_vectors(6), oracle.hop_vectors(14)
    assert np.array_equal(v14[:6], v6)
    assert sorted(map(tuple, v6.tolist())) == sorted(faces)
    for a in range(3):  # +axis then -axis, x before y before z
        assert tuple(v6[2 * a]) == tuple(int(a == b) for b in range(3))
        assert tuple(v6[2 * a + 1]) == tuple(-int(a == b) for b in range(3))
    assert sorted(map(tuple, v14[6:].tolist())) == sorted(diag)
    # x fastest, + before -: the sign pattern counts in binary with x as the low bit
    code = [(v[0] < 0) + 2 * (v[1] < 0) + 4 * (v[2] < 0) for v in v14[6:].tolist()]
    assert code == list(range(8))
    E = 5
    s = np.arange(E ** 3)
    xyz = workloads.site_xyz(E, s)
    for nh, V in ((6, v6), (14, v14)):
        t = oracle.hop_targets(E, s, nh)
        for k in range(nh):
            w = (xyz + V[k]) % E
            assert np.array_equal(t[:, k], w[:, 0] + E * (w[:, 1] + E * w[:, 2]))
            assert all(oracle.hop_target(E, int(x), k) == int(t[x, k]) for x in (0, E - 1, E ** 3 - 1))


def test_masks_mark_occupied_targets():
    E = 4
    sites, q = workloads.random_small(E, 30, 19)  # dense: many blocked hops
    st = oracle.LatticeState(E, sites, q)
    dU, mask = st.propose()
    occ = set(sites.tolist())
    for i in range(st.n):
        for k in range(6):
            blocked = st.target(i, k) in occ
            assert mask[i, k] == (0 if blocked else 1)
            assert np.isnan(dU[i, k]) == blocked


# ------------------------------------------------------------------ KMC step
def _numpy_select(rate, zeta):
    R = np.cumsum(rate)
    Q = R[-1]
    j = int(np.searchsorted(R, Q * zeta, side="left"))
    return j, Q


def test_selection_matches_independent_version():
    rng = np.random.default_rng(23)
    for trial in range(200):
        m = int(rng.integers(1, 60))
        rate = rng.random(m)
        rate[rng.random(m) < 0.3] = 0.0
        if trial % 7 == 0:
            rate[:] = 0.5  # exact ties in the cumulative sums
        if rate.sum() == 0:
            rate[0] = 1.0
        zeta = 1.0 - rng.random()
        if trial % 11 == 0:
            zeta = 1.0
        j, Q, dt = oracle.select(rate, zeta, 0.5)
        j2, Q2 = _numpy_select(rate, zeta)
        assert Q == Q2
        assert j == j2
        assert rate[j] > 0.0
        assert abs(dt + math.log(0.5) / Q) < 1e-15 * abs(dt) + 1e-300


def test_selection_chi_square():
    rate = np.array([0.1, 0.0, 2.0, 0.5, 0.5, 1.0, 0.0, 3.9])
    rng = np.random.default_rng(29)
    n = 200_000
    counts = np.zeros(len(rate))
    R = oracle.cumsum(rate)
    Q = R[-1]
    # the same rule applied vectorised to many draws, cross-checked on a subset
    z = 1.0 - rng.random(n)
    js = np.searchsorted(R, Q * z, side="left")
    for t in range(0, n, 4000):
        assert oracle.select(rate, float(z[t]), 0.5)[0] == js[t]
    np.add.at(counts, js, 1)
    p = rate / Q
    ok = p > 0
    assert counts[~ok].sum() == 0
    chi2 = float(np.sum((counts[ok] - n * p[ok]) ** 2 / (n * p[ok])))
    # 5 degrees of freedom: P(chi2 > 25) ~ 1.4e-4
    assert chi2 < 25.0, chi2


def test_rates_rule():
    dU = np.array([-1.0, 0.0, 0.05, 0.5, np.nan])
    mask = np.array([1, 1, 1, 1, 0], dtype=np.uint8)
    r = oracle.rates(dU, mask, 0.05)
    assert np.allclose(r, [1.0, 1.0, math.exp(-1.0), math.exp(-10.0), 0.0], rtol=1e-15, atol=0)


def test_kmc_step_moves_charge():
    st = _state(8, 40, 31)
    before = st.sites.copy()
    j, dt, Q, dU, mask = oracle.kmc_step(st, 0.1, 0.37, 0.5)
    i, k = j // 6, j % 6
    assert mask[i, k] == 1
    assert st.sites[i] == oracle.hop_target(8, int(before[i]), k)
    assert np.array_equal(np.delete(st.sites, i), np.delete(before, i))


# ---------------------------------------------------------------- free space
def test_free_two_charges_closed_form():
    """+1 at the origin moved to (1,0,0) next to -1 at (3,0,0): dU = -(1/2 - 1/3) = -1/6."""
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    q = np.array([1.0, -1.0])
    du = oracle.free_delta_u(pos, q, [0], [[1.0, 0.0, 0.0]])[0]
    assert abs(du - (-1.0 / 6.0)) < 1e-15
    assert abs(oracle.free_energy(pos, q) - (-1.0 / 3.0)) < 1e-15


def test_free_square_energy_closed_form():
    """Alternating +-1 on the corners of a unit square: four bonds of -1 and
    two diagonals of +1/sqrt(2): U = -4 + sqrt(2)."""
    pos = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=float)
    q = np.array([1.0, -1.0, 1.0, -1.0])
    assert abs(oracle.free_energy(pos, q) - (-4.0 + math.sqrt(2.0))) < 1e-14


def test_free_delta_u_equals_energy_difference():
    rng = np.random.default_rng(11)
    pos = rng.random((40, 3)) * 10.0
    q = rng.choice([-1.0, 1.0, 2.0], size=40)  # free space: no neutrality needed
    U0 = oracle.free_energy(pos, q)
    for k in range(5):
        t = rng.random(3) * 10.0
        du = oracle.free_delta_u(pos, q, [k], [t])[0]
        p2 = pos.copy()
        p2[k] = t
        assert abs(du - (oracle.free_energy(p2, q) - U0)) < 1e-12 * max(1.0, abs(U0))


def test_free_hop_reverse_and_rigid_motion():
    rng = np.random.default_rng(12)
    pos = rng.random((30, 3)) * 8.0
    q = rng.choice([-1.0, 1.0], size=30)
    t = pos[3] + np.array([1.0, 0.0, 0.0])
    du1 = oracle.free_delta_u(pos, q, [3], [t])[0]
    p2 = pos.copy()
    p2[3] = t
    du2 = oracle.free_delta_u(p2, q, [3], [pos[3]])[0]
    assert abs(du1 + du2) < 1e-13
    # translation and a rotation by 90 degrees about z leave dU unchanged
    shift = np.array([3.5, -2.0, 7.25])
    assert abs(oracle.free_delta_u(pos + shift, q, [3], [t + shift])[0] - du1) < 1e-12
    rot = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    assert abs(oracle.free_delta_u(pos @ rot.T, q, [3], [rot @ t])[0] - du1) < 1e-12


def test_free_singular_targets():
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = np.array([1.0, -1.0])
    out = oracle.free_delta_u(pos, q, [0, 0], [[1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert np.isnan(out).all()


# ---------------------------------------------------------------- Dirichlet walls
def _dirichlet_system(E, n, seed):
    rng = np.random.default_rng(seed)
    half = np.arange(E ** 3)[np.arange(E ** 3) // (E * E) < E // 2]
    sites = rng.choice(half, n, replace=False)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    return sites, q


def test_dirichlet_potential_vanishes_on_both_walls():
    """The mirrored cell's potential is zero on z = 0 and on z = a/2 (grounded walls)."""
    E = 6
    sites, q = _dirichlet_system(E, 8, 31)
    st = oracle.DirichletLattice(E, sites, q, oracle.hop_vectors(6))
    pos = workloads.site_positions(E, st.ext.sites)
    a = float(E)
    rng = np.random.default_rng(5)
    for zw in (0.0, a / 2):
        for _ in range(3):
            x = np.array([rng.random() * a, rng.random() * a, zw])
            phi = sum(st.ext.q[j] * oracle.psi(a, x - pos[j]) for j in range(len(st.ext.q)))
            assert abs(phi) < 1e-12


def test_dirichlet_hop_energy_equals_brute_force():
    """dU of every allowed hop equals half the brute-force Ewald energy change of
    the mirrored cell when the charge and its mirror move, plus the field term."""
    E, fz = 6, 0.3
    sites, q = _dirichlet_system(E, 10, 32)
    st = oracle.DirichletLattice(E, sites, q, oracle.hop_vectors(14), field_z=fz)
    dU, mask = st.propose()
    a = float(E)
    pos0 = workloads.site_positions(E, st.ext.sites)
    U0 = oracle.energy(pos0, st.ext.q, a)
    assert abs(st.energy() - (0.5 * U0 - fz * np.dot(q, pos0[:10, 2]))) < 1e-12
    checked = 0
    for i in (0, 3, 7):
        for k in range(14):
            if not mask[i, k]:
                continue
            t = oracle.hop_targets(E, st.sites[i:i + 1], 14)[0, k]
            s2 = st.ext.sites.copy()
            s2[i] = t
            s2[i + 10] = oracle.mirror_sites(E, np.array([t]))[0]
            U1 = oracle.energy(workloads.site_positions(E, s2), st.ext.q, a)
            dz = (t // (E * E)) - (st.sites[i] // (E * E))
            assert abs(dU[i, k] - (0.5 * (U1 - U0) - q[i] * fz * dz)) < 1e-11, (i, k)
            checked += 1
    assert checked >= 10
    # hops through a wall are masked
    zs = st.sites // (E * E)
    for i in range(10):
        for k, hv in enumerate(oracle.hop_vectors(14)):
            if zs[i] + hv[2] < 0 or zs[i] + hv[2] >= E // 2:
                assert not mask[i, k]
