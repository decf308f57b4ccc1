"""Pins of the oracle's arithmetic against what the mathematics fixes.

Each test would fail for a plausible slip in the oracle: a dropped or mis-signed
term breaks energy neutrality or skewness; a wrong stride offset breaks the
Table-"Communication aggregation" patterns, the closed forms or the mirror
symmetries; a wrong integrator breaks the amplification polynomial.
The weights of the energy inner product are written here from their closed
form (reading R4), independently of the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import TERM_ADV, TERM_ALL, TERM_COR, TERM_PGF_PHI, TERM_PGF_PI
from paper_2103_10114_gb300 import inputs

A_E = 6.371e6
RT0 = 287.04 * 250.0
FIELDS = ("U", "V", "Phi", "pi")


def weights(I, J, K, phis, sigma_half=None):
    dl, dth = 2 * math.pi / I, math.pi / J
    s = np.sin((np.arange(J) + 0.5) * dth)
    sv = np.sin((np.arange(J - 1) + 1.0) * dth)
    A = A_E**2 * s * dth * dl
    Av = A_E**2 * sv * dth * dl
    sh = np.arange(K + 1) / K if sigma_half is None else np.asarray(sigma_half)
    ds = np.diff(sh)
    pit = np.exp(-np.asarray(phis) / RT0)
    return {
        "U": ds[:, None, None] * A[None, :, None] * np.ones((K, J, I)),
        "V": ds[:, None, None] * Av[None, :, None] * np.ones((K, J - 1, I)),
        "Phi": ds[:, None, None] * A[None, :, None] * np.ones((K, J, I)),
        "pi": A[:, None] * RT0 / pit,
    }


def inner(w, x, y):
    return sum(float(np.sum(w[f] * x[f] * y[f])) for f in FIELDS)


def absinner(w, x, y):
    return sum(float(np.sum(w[f] * np.abs(x[f] * y[f]))) for f in FIELDS)


def state_only(st):
    return {f: st[f] for f in FIELDS}


GRIDS = [
    dict(I=16, J=10, K=4),  # default Eq. 7 table, strides up to 5
    dict(I=12, J=8, K=3, sig=[0.0, 0.1, 0.45, 1.0]),  # non-uniform sigma
    dict(I=20, J=9, K=5, rand_leap=True),  # random odd table, odd nlat
]


def make(g, seed):
    I, J, K = g["I"], g["J"], g["K"]
    st = inputs.random_state(I, J, K, seed=seed)
    mu = mv = None
    if g.get("rand_leap"):
        rng = np.random.default_rng(seed + 100)
        mu = 2 * rng.integers(0, (I - 1) // 4 + 1, J) + 1
        mv = 2 * rng.integers(0, (I - 1) // 4 + 1, J - 1) + 1
    o = oracle.Oracle(I, J, K, sigma_half=g.get("sig"), leap_u=mu, leap_v=mv, phis=st["phis"])
    w = weights(I, J, K, st["phis"], g.get("sig"))
    return o, st, w


@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("terms", [TERM_ADV, TERM_COR, TERM_PGF_PI, TERM_PGF_PHI, TERM_ALL])
def test_I1_energy_neutral(gi, terms):
    """<x, T(x)>_W = 0: exact semi-discrete energy conservation, per term group."""
    o, st, w = make(GRIDS[gi], seed=10 + gi)
    t = o.tendency(st, terms)
    assert abs(inner(w, st, t)) <= 1e-13 * absinner(w, st, t)
    assert absinner(w, st, t) > 0


@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_I2_mass(gi):
    o, st, w = make(GRIDS[gi], seed=20 + gi)
    t = o.tendency(st)
    A = w["pi"] * np.exp(-st["phis"] / RT0) / RT0  # area weights
    assert abs(np.sum(A * t["pi"])) <= 1e-14 * np.sum(A * np.abs(t["pi"]))


def test_energy_pin_catches_a_planted_error():
    """The energy pin is sensitive: halving one Coriolis branch breaks it."""
    o, st, w = make(GRIDS[0], seed=3)
    t = o.tendency(st, TERM_COR)
    tu_only = dict(t)
    tu_only["V"] = 0.5 * t["V"]
    assert abs(inner(w, st, tu_only)) > 1e-6 * absinner(w, st, tu_only)


def test_rest_state_over_terrain_stays_at_rest():
    """U = V = Phi = pi = 0 over any terrain: the standard atmosphere is balanced."""
    I, J, K = 16, 10, 4
    st = inputs.random_state(I, J, K, seed=5)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    t = o.tendency(o.zeros())
    assert max(np.abs(v).max() for v in t.values()) == 0.0


@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_I3_linearisation_about_rest_is_skew(gi):
    """About rest the operator is linear (PGF/divergence pair, Coriolis with
    f = 2 Omega cos, hydrostatic/Omega~ pair, dpi/dt); it is W-skew:
    <y, J x>_W = -<J y, x>_W for random x, y."""
    o, st, w = make(GRIDS[gi], seed=30 + gi)
    I, J, K = GRIDS[gi]["I"], GRIDS[gi]["J"], GRIDS[gi]["K"]
    x = state_only(inputs.random_state(I, J, K, seed=31, terrain=False))
    y = state_only(inputs.random_state(I, J, K, seed=32, terrain=False))
    rest = o.zeros()
    Jx, Jy = o.tendency_jvp(rest, x), o.tendency_jvp(rest, y)
    lhs, rhs = inner(w, y, Jx), inner(w, Jy, x)
    assert abs(lhs + rhs) <= 1e-13 * (absinner(w, y, Jx) + absinner(w, Jy, x))


def test_jvp_matches_central_differences():
    o, st, w = make(GRIDS[0], seed=40)
    I, J, K = 16, 10, 4
    d = inputs.random_direction(I, J, K)
    jv = o.tendency_jvp(st, d)
    h = 1e-5
    tp = o.tendency({f: st[f] + h * d[f] for f in FIELDS})
    tm = o.tendency({f: st[f] - h * d[f] for f in FIELDS})
    for f in FIELDS:
        fd = (tp[f] - tm[f]) / (2 * h)
        assert np.abs(fd - jv[f]).max() <= 1e-6 * np.abs(jv[f]).max(), f


# ---- Table "Communication aggregation" patterns, assembled from index lists ----

def _jac_block(o, out_field, in_field, terms=TERM_ALL):
    """Columns of dT[out]/dx[in] at rest (flat terrain), one JVP per unit vector."""
    sh = o.shapes()
    n_in = int(np.prod(sh[in_field]))
    cols = []
    for q in range(n_in):
        d = o.zeros()
        d[in_field].reshape(-1)[q] = 1.0
        cols.append(o.tendency_jvp(o.zeros(), d, terms)[out_field].reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("ones", [False, True])
def test_leap_divergence_and_gradient_patterns(ones):
    """Divergence: the (x+N-1, x-N) pair, gradient: the (x+N, x-N+1) pair of
    Table "Communication aggregation", with N = (M+1)/2, over a sin(theta) M dlam
    (Eq. 6; Eq. 5 when every M = 1)."""
    I, J, K = 14, 8, 2
    mu = np.ones(J, np.int32) if ones else None
    mv = np.ones(J - 1, np.int32) if ones else None
    o = oracle.Oracle(I, J, K, leap_u=mu, leap_v=mv)
    dl, dth = 2 * math.pi / I, math.pi / J
    s = np.sin((np.arange(J) + 0.5) * dth)
    M = o.leap_u
    if ones:
        assert np.all(M == 1)
    else:
        assert M.max() > 1
    # divergence from the U block of dpi/dt at rest: dpi/dt = -sum_k ds_k D(U_k)
    Jpu = _jac_block(o, "pi", "U")  # (J*I, K*J*I)
    Dm = np.zeros((J * I, J * I))
    Gm = np.zeros((J * I, J * I))
    for j in range(J):
        N = (M[j] + 1) // 2
        c = 1.0 / (A_E * s[j] * M[j] * dl)
        for x in range(I):
            Dm[j * I + x, j * I + (x + N - 1) % I] += c
            Dm[j * I + x, j * I + (x - N) % I] -= c
            Gm[j * I + x, j * I + (x + N) % I] += c
            Gm[j * I + x, j * I + (x - N + 1) % I] -= c
    ds = 1.0 / K
    for k in range(K):
        blk = Jpu[:, k * J * I:(k + 1) * J * I]
        assert np.allclose(blk, -ds * Dm, rtol=0, atol=1e-12 * np.abs(Dm).max())
    # gradient from the pi block of dU/dt at rest: dU/dt = -R T0 G(pi)
    Jup = _jac_block(o, "U", "pi")
    for k in range(K):
        blk = Jup[k * J * I:(k + 1) * J * I, :]
        assert np.allclose(blk, -RT0 * Gm, rtol=0, atol=1e-12 * RT0 * np.abs(Gm).max())


@pytest.mark.parametrize("ones", [False, True])
def test_centred_advection_pattern(ones):
    """Uniform zonal flow c over flat ground advects Phi with the centred
    (x + 2N-1, x - 2N+1) = x +- M pair: dPhi/dt = -c (Phi[i+M] - Phi[i-M]) / (2 a sin M dlam)."""
    I, J, K = 18, 8, 2
    mu = np.ones(J, np.int32) if ones else None
    mv = np.ones(J - 1, np.int32) if ones else None
    o = oracle.Oracle(I, J, K, leap_u=mu, leap_v=mv)
    dl, dth = 2 * math.pi / I, math.pi / J
    s = np.sin((np.arange(J) + 0.5) * dth)
    st = o.zeros()
    c = 7.0
    st["U"][:] = c
    st["Phi"] = np.random.default_rng(1).normal(0, 10, st["Phi"].shape)
    t = o.tendency(st)
    M = o.leap_u
    for j in range(J):
        P = st["Phi"][:, j, :]
        want = -c * (np.roll(P, -M[j], axis=1) - np.roll(P, M[j], axis=1)) / (2 * A_E * s[j] * M[j] * dl)
        assert np.allclose(t["Phi"][:, j, :], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


# ---- I5: closed forms of the stride-M operators on e^{i n lambda} --------------

@pytest.mark.parametrize("n", [1, 3, 5])
def test_I5_closed_forms(n):
    I, J, K = 24, 12, 1
    o = oracle.Oracle(I, J, K)
    dl, dth = 2 * math.pi / I, math.pi / J
    s = np.sin((np.arange(J) + 0.5) * dth)
    lam = np.arange(I) * dl
    M = o.leap_u[:, None]
    # staggered: U = cos(n lambda_{u+1/2}), P = 1  ->  dpi/dt = -D
    st = o.zeros()
    st["U"][0] = np.cos(n * (lam + 0.5 * dl))[None, :]
    t = o.tendency(st, TERM_PGF_PI)
    want = 2 * np.sin(n * lam)[None, :] * np.sin(n * M * dl / 2) / (A_E * s[:, None] * M * dl)
    assert np.allclose(t["pi"], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    # centred: uniform U = c carries Phi = cos(n lambda)
    st = o.zeros()
    c = 3.0
    st["U"][:] = c
    st["Phi"][0] = np.cos(n * lam)[None, :]
    t = o.tendency(st, TERM_ADV)
    want = c * np.sin(n * lam)[None, :] * np.sin(n * M * dl) / (A_E * s[:, None] * M * dl)
    assert np.allclose(t["Phi"][0], want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


# ---- mirror symmetries ------------------------------------------------------------

def _mirror_lon(st, I):
    sc = (-np.arange(I)) % I  # scalar/V index i -> -i
    uu = (I - 1 - np.arange(I))  # U index u (lambda_{u+1/2}) -> I-1-u
    out = {"U": -st["U"][..., uu], "V": st["V"][..., sc], "Phi": st["Phi"][..., sc], "pi": st["pi"][..., sc]}
    if "phis" in st:
        out["phis"] = st["phis"][..., sc]
    return out


def _mirror_lat(st):
    out = {"U": st["U"][:, ::-1, :], "V": -st["V"][:, ::-1, :], "Phi": st["Phi"][:, ::-1, :],
           "pi": st["pi"][::-1, :]}
    if "phis" in st:
        out["phis"] = st["phis"][::-1, :]
    return out


def test_zonal_mirror_symmetry():
    """lambda -> -lambda (U -> -U) commutes with the operator without the
    planetary rotation (which flips sign under the mirror)."""
    I, J, K = 16, 10, 3
    st = inputs.random_state(I, J, K, seed=50)
    terms = TERM_ADV | TERM_PGF_PI | TERM_PGF_PHI
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    t = o.tendency(st, terms)
    ms = _mirror_lon(st, I)
    om = oracle.Oracle(I, J, K, phis=ms["phis"])
    tm = om.tendency(ms, terms)
    mt = _mirror_lon(t, I)
    for f in FIELDS:
        assert np.allclose(tm[f], mt[f], rtol=1e-11, atol=1e-11 * np.abs(t[f]).max()), f


def test_meridional_mirror_symmetry():
    """theta -> pi - theta (V -> -V) commutes with the whole operator."""
    I, J, K = 16, 10, 3
    st = inputs.random_state(I, J, K, seed=51)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    assert np.array_equal(o.leap_u, o.leap_u[::-1]) and np.array_equal(o.leap_v, o.leap_v[::-1])
    t = o.tendency(st)
    ms = _mirror_lat(st)
    om = oracle.Oracle(I, J, K, phis=ms["phis"])
    tm = om.tendency(ms)
    mt = _mirror_lat(t)
    for f in FIELDS:
        assert np.allclose(tm[f], mt[f], rtol=1e-10, atol=1e-10 * np.abs(t[f]).max()), f


# ---- I6: brute force on tiny grids ---------------------------------------------------

def _full_jacobian(o, st, fn):
    sh = o.shapes()
    sizes = [int(np.prod(sh[f])) for f in FIELDS]
    cols = []
    for fi, f in enumerate(FIELDS):
        for q in range(sizes[fi]):
            d = o.zeros()
            d[f].reshape(-1)[q] = 1.0
            out = fn(st, d)
            cols.append(np.concatenate([out[g].reshape(-1) for g in FIELDS]))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims", [(8, 6, 2), (10, 6, 3)])
def test_I6_spectrum_and_amplification(dims):
    I, J, K = dims
    st = inputs.random_state(I, J, K, seed=60)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    rest = o.zeros()
    Jm = _full_jacobian(o, rest, lambda s, d: o.tendency_jvp(s, d))
    w = weights(I, J, K, st["phis"])
    Wd = np.concatenate([w[f].reshape(-1) for f in FIELDS])
    # skew in W: W J + J^T W = 0
    S = Wd[:, None] * Jm
    assert np.abs(S + S.T).max() <= 1e-12 * np.abs(S).max()
    ev = np.linalg.eigvals(Jm)
    assert np.abs(ev.real).max() <= 1e-9 * np.abs(ev).max()
    # one step about rest is the polynomial 1 + z + z^2/2 + z^3/4 of dt J (reading R9)
    dt = 0.7 / np.abs(ev).max()
    Sm = _full_jacobian(o, rest, lambda s, d: o.step_jvp(s, d, dt, 1)[1])
    Z = dt * Jm
    Id = np.eye(Z.shape[0])
    poly = Id + Z + Z @ Z / 2 + Z @ Z @ Z / 4
    assert np.abs(Sm - poly).max() <= 1e-12 * np.abs(poly).max()
    # and each eigenmode's amplification has modulus <= 1 for |z| <= 2
    amp = np.abs(1 + dt * ev + (dt * ev) ** 2 / 2 + (dt * ev) ** 3 / 4)
    assert np.all(amp <= 1 + 1e-12)


# ---- I8: energy loss of the three-stage step is O(dt^3) over a fixed time ----------

def test_I8_energy_drift_order():
    I, J, K = 32, 16, 3
    st = inputs.rossby_haurwitz4(I, J, K, seed=7)
    o = oracle.Oracle(I, J, K)
    e0 = o.diagnostics(st)["energy"]
    T = 4 * 600.0
    drift = []
    for n in (4, 8, 16):
        x = o.step(st, T / n, n)
        drift.append(e0 - o.diagnostics(x)["energy"])
    assert all(d > 0 for d in drift)  # the scheme only loses energy
    r1, r2 = drift[0] / drift[1], drift[1] / drift[2]
    assert 6.0 < r1 < 10.5 and 6.5 < r2 < 9.5, (r1, r2)


def test_mass_conserved_over_steps():
    I, J, K = 32, 16, 3
    st = inputs.baroclinic_jet(I, J, K, seed=8, terrain_seed=2)
    o = oracle.Oracle(I, J, K, phis=st["phis"])
    m0 = o.diagnostics(st)["mass"]
    x = o.step(st, 300.0, 5)
    assert abs(o.diagnostics(x)["mass"] / m0 - 1) < 1e-13


def test_rejects_bad_tables():
    with pytest.raises(ValueError):
        oracle.Oracle(16, 8, 2, leap_u=np.full(8, 2))  # even stride
    with pytest.raises(ValueError):
        oracle.Oracle(16, 8, 2, leap_u=np.full(8, 9))  # 2M >= nlon
    with pytest.raises(ValueError):
        oracle.Oracle(16, 8, 2, sigma_half=[0.0, 0.6, 0.5])  # non-monotone sigma


def test_operation_count_is_faithful_and_stride_free():
    """The counting type changes no result, and its tally is the same per grid
    point whatever the leap strides (doubling nlon changes every stride)."""
    counts = []
    for I in (32, 64):
        J, K = 16, 4
        st = inputs.random_state(I, J, K, seed=5)
        o = oracle.Oracle(I, J, K, phis=st["phis"])
        t, ops = o.tendency_opcount(st)
        t0 = o.tendency(st)
        assert all(np.array_equal(t[f], t0[f]) for f in t0)
        assert min(ops.values()) > 0
        counts.append(ops)
    assert all(counts[1][k] == 2 * counts[0][k] for k in counts[0])


@pytest.mark.parametrize("shift", [1, 3, 7])
def test_zonal_translation_invariance(shift):
    """Every longitude is treated alike: shifting all fields (U keeps its half
    point offset) by s grid points shifts the tendency by s, bit for bit,
    including across the periodic seam; random odd strides up to nlon/2 make
    every leap offset wrap somewhere."""
    I, J, K = 20, 9, 4
    rng = np.random.default_rng(3)
    mu = 2 * rng.integers(0, 5, J) + 1
    mv = 2 * rng.integers(0, 5, J - 1) + 1
    st = inputs.random_state(I, J, K, seed=8)
    phis = np.asarray(st["phis"]).reshape(J, I)
    o = oracle.Oracle(I, J, K, leap_u=mu, leap_v=mv, phis=phis)
    o_s = oracle.Oracle(I, J, K, leap_u=mu, leap_v=mv, phis=np.roll(phis, shift, axis=-1))
    x = state_only(st)
    xs = {f: np.roll(v, shift, axis=-1) for f, v in x.items()}
    t, ts = o.tendency(x), o_s.tendency(xs)
    for f in FIELDS:
        assert np.array_equal(np.roll(t[f], shift, axis=-1), ts[f]), f
