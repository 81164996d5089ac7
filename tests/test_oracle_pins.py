"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: brute force with
exact rational arithmetic, closed forms of hand-built fields, the mesh rebuilt
from the paper's prism split, optimality of Huffman codes, library logarithms.
"""
import heapq
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2510_25143_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Simulation of Simplicity (Sec. III-F, Alg. 1) and the face test (Eqs. 1-3)
# ---------------------------------------------------------------------------
def _solve3(A, b):
    """Gaussian elimination over Fractions (no pivoting shortcuts)."""
    M = [list(A[r]) + [b[r]] for r in range(3)]
    for c in range(3):
        p = next(r for r in range(c, 3) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(3):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][k] - f * M[c][k] for k in range(4)]
    return [M[r][3] / M[r][r] for r in range(3)]


def _inside_perturbed(vals, eps=Fraction(1, 1000)):
    """Origin strictly inside conv of the three perturbed values: solve Eq. 1
    ([u;v;1] mu = [0;0;1]) exactly for the SoS-perturbed vertex values, the
    vertex of rank r moved by (eps^(2^(2r-1)), eps^(2^(2r-2)))."""
    pts = []
    for r in range(1, 4):
        u, v = vals[2 * (r - 1)], vals[2 * (r - 1) + 1]
        pts.append((Fraction(u) + eps ** (2 ** (2 * r - 1)), Fraction(v) + eps ** (2 ** (2 * r - 2))))
    A = [[p[0] for p in pts], [p[1] for p in pts], [Fraction(1)] * 3]
    mu = _solve3(A, [Fraction(0), Fraction(0), Fraction(1)])
    return all(m > 0 for m in mu)


def test_sos_predicate_exhaustive_small_domain():
    """All 5^6 faces with values in {-2..2}: the SoS predicate equals the exact
    barycentric solve of the symbolically perturbed triangle."""
    cases = np.array(list(itertools.product(range(-2, 3), repeat=6)), np.int64)
    got = oracle.face_crossed_batch(cases)
    want = np.array([_inside_perturbed(tuple(int(x) for x in c)) for c in cases])
    assert got.sum() > 0
    assert (got == want).all(), np.nonzero(got != want)[0][:10]


def test_face_test_nondegenerate_matches_barycentric():
    """Away from degeneracies the predicate is Eq. 2 / Eq. 3: origin inside iff
    all barycentric coordinates of the origin are positive."""
    rng = np.random.default_rng(7)
    p = rng.integers(-10**6, 10**6, (4000, 6))
    got = oracle.face_crossed_batch(p)
    for c, g in zip(p, got):
        pts = [(int(c[0]), int(c[1])), (int(c[2]), int(c[3])), (int(c[4]), int(c[5]))]
        A = [[Fraction(x[0]) for x in pts], [Fraction(x[1]) for x in pts], [Fraction(1)] * 3]
        mu = _solve3(A, [Fraction(0), Fraction(0), Fraction(1)])
        assert all(m != 0 for m in mu)
        assert g == all(m > 0 for m in mu)
    assert 0 < got.sum() < len(got)


# ---------------------------------------------------------------------------
# Mesh (Sec. III-C): rebuild faces and tets from the paper's prism split
# ---------------------------------------------------------------------------
def _paper_mesh(H, W, T):
    """Faces and tets of the extruded mesh built directly from the paper:
    triangles of the main-diagonal triangulation, each prism [t,t+1] split into
    tau1=(a_t,b_t,c_t,c_t+1), tau2=(a_t,b_t,b_t+1,c_t+1), tau3=(a_t,a_t+1,b_t+1,c_t+1)
    with a<b<c by vertex id."""
    def vid(t, i, j):
        return (t * H + i) * W + j
    tris = []
    for i in range(H - 1):
        for j in range(W - 1):
            tris.append(sorted([(i, j), (i, j + 1), (i + 1, j + 1)], key=lambda p: p[0] * W + p[1]))
            tris.append(sorted([(i, j), (i + 1, j), (i + 1, j + 1)], key=lambda p: p[0] * W + p[1]))
    faces, tets = set(), []
    for t in range(T):
        for a, b, c in tris:
            faces.add(tuple(sorted((vid(t, *a), vid(t, *b), vid(t, *c)))))
    for t in range(T - 1):
        for a, b, c in tris:
            A0, B0, C0 = vid(t, *a), vid(t, *b), vid(t, *c)
            A1, B1, C1 = vid(t + 1, *a), vid(t + 1, *b), vid(t + 1, *c)
            for tet in ((A0, B0, C0, C1), (A0, B0, B1, C1), (A0, A1, B1, C1)):
                fs = [tuple(sorted(f)) for f in itertools.combinations(tet, 3)]
                tets.append(frozenset(fs))
                faces.update(fs)
    return faces, tets


def _oracle_mesh(H, W, T):
    F = oracle.face_table()
    TT = oracle.tet_table()

    def vid(t, i, j):
        return (t * H + i) * W + j

    def face_vertices(t, i, j, ty):
        return tuple(sorted(vid(t + F[ty][k][0], i + F[ty][k][1], j + F[ty][k][2]) for k in range(3)))

    def valid(t, i, j, ty):
        return all(t + F[ty][k][0] < T and i + F[ty][k][1] < H and j + F[ty][k][2] < W for k in range(3))

    faces = set()
    for t in range(T):
        for i in range(H):
            for j in range(W):
                for ty in range(12):
                    if valid(t, i, j, ty):
                        faces.add(face_vertices(t, i, j, ty))
    tets = []
    for t in range(T - 1):
        for i in range(H - 1):
            for j in range(W - 1):
                for k in range(6):
                    tets.append(frozenset(face_vertices(t + e[0], i + e[1], j + e[2], e[3]) for e in TT[k]))
    return faces, tets


def test_mesh_tables_match_paper_split():
    for H, W, T in [(4, 5, 3), (6, 6, 4)]:
        pf, pt = _paper_mesh(H, W, T)
        of, ot = _oracle_mesh(H, W, T)
        assert pf == of
        assert sorted(map(sorted, pt)) == sorted(map(sorted, ot))
        assert oracle.face_count(H, W, T) == len(pf)


def test_mesh_counts_golden():
    """Closed-form face and tet counts (Sec. III-C extrusion), incl. 1010 faces on 6x6x4."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "mesh_counts.txt")) if l[0] != "#"]
    for H, W, T, faces, tets in [tuple(map(int, r)) for r in rows]:
        E = H * (W - 1) + W * (H - 1) + (H - 1) * (W - 1)
        assert faces == 2 * (H - 1) * (W - 1) * T + (T - 1) * (2 * E + 4 * (H - 1) * (W - 1))
        assert tets == 6 * (H - 1) * (W - 1) * (T - 1)
        if H * W * T <= 64 * 64 * 8:
            assert oracle.face_count(H, W, T) == faces


def test_incident_faces_36():
    """An interior vertex lies on 36 faces (Alg. 4 / Sec. V-B), fewer on the boundary."""
    H, W, T = 6, 7, 5
    _, _ = H, W
    pf, _ = _paper_mesh(H, W, T)
    for t in range(T):
        for i in range(H):
            for j in range(W):
                v = (t * H + i) * W + j
                n = sum(v in f for f in pf)
                assert oracle.incident_face_count(H, W, T, t, i, j) == n
                if 0 < t < T - 1 and 0 < i < H - 1 and 0 < j < W - 1:
                    assert n == 36


# ---------------------------------------------------------------------------
# Lemma 1: every tet has 0 or 2 crossed faces under SoS
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_lemma1_parity_small_integer_fields(seed):
    rng = np.random.default_rng(seed)
    uv = rng.integers(-2, 3, (4, 5, 6, 2)).astype(np.float32)
    q = oracle.to_fixed(uv, oracle.scale_exponent(np.abs(uv).max()))
    _, _, bad = oracle.trajectories(q)
    assert bad == 0


def test_lemma1_parity_vortex64():
    uv = synth.vortex_sum()
    k = oracle.scale_exponent(np.abs(uv).max())
    trajs, _, bad = oracle.trajectories(oracle.to_fixed(uv, k))
    assert bad == 0 and len(trajs) > 0


# ---------------------------------------------------------------------------
# Hand-built fields with known zero paths (Sec. III-D, Thm. 1, Eq. 3)
# ---------------------------------------------------------------------------
def _slice_cps(mask):
    return ((mask & 1) > 0).sum(axis=(1, 2)) + ((mask & 2) > 0).sum(axis=(1, 2))


@pytest.mark.parametrize("saddle", [False, True])
def test_linear_field_single_trajectory(saddle):
    H, W, T = 24, 32, 8
    a, b, c, d = 6.3, 1.7, 5.6, 1.45
    uv = synth.linear_field(H, W, T, a, b, c, d, saddle=saddle)
    k = oracle.scale_exponent(np.abs(uv).max())
    q = oracle.to_fixed(uv, k)
    m = oracle.face_masks(q)
    assert (_slice_cps(m) == 1).all()
    trajs, pts, bad = oracle.trajectories(q)
    assert bad == 0 and len(trajs) == 1
    # crossing points on slice faces sit exactly on x = a + b t, y = c + d t
    F = oracle.face_table()
    for fid, p in zip(trajs[0], pts[0]):
        ty = int(fid % 12)
        if ty < 2:
            t = p[2]
            assert abs(p[0] - (a + b * t)) < 1e-5 and abs(p[1] - (c + d * t)) < 1e-5
    assert F.shape == (12, 3, 3)


def _face_triples(fids, H, W):
    F = oracle.face_table()
    out = []
    for fid in fids:
        owner, ty = divmod(int(fid), 12)
        t, rem = divmod(owner, H * W)
        i, j = divmod(rem, W)
        out.append(tuple(sorted(((t + F[ty][k][0]) * H + i + F[ty][k][1]) * W + j + F[ty][k][2]
                                for k in range(3))))
    return out


@pytest.mark.parametrize("case", ["smooth_noise", "small_ints"])
def test_trajectories_are_the_components_of_crossed_faces(case):
    """R13 by brute force: the trajectories are the connected components of
    the crossed faces, two faces joined when they bound one tetrahedron of the
    prism split (the mesh rebuilt here from the paper), each listed as a path
    whose consecutive faces share a tetrahedron."""
    if case == "smooth_noise":  # many critical points: smoothed Gaussian noise
        from scipy.ndimage import gaussian_filter
        r = np.random.default_rng(31).normal(size=(5, 16, 18, 2))
        uv = gaussian_filter(r, (0.8, 1.5, 1.5, 0)).astype(np.float32)
    else:
        uv = np.random.default_rng(32).integers(-2, 3, (4, 7, 8, 2)).astype(np.float32)
    T, H, W, _ = uv.shape
    k = oracle.scale_exponent(np.abs(uv).max())
    q = oracle.to_fixed(uv, k)
    trajs, _, bad = oracle.trajectories(q)
    assert bad == 0
    m = oracle.face_masks(q)
    crossed = set()
    for owner in np.flatnonzero(m.reshape(-1)):
        for ty in range(12):
            if (int(m.reshape(-1)[owner]) >> ty) & 1:
                crossed.add(_face_triples([owner * 12 + ty], H, W)[0])
    _, tets = _paper_mesh(H, W, T)
    adj = {f: set() for f in crossed}
    for tet in tets:
        hit = [f for f in tet if f in crossed]
        assert len(hit) in (0, 2)  # Lemma 1
        if hit:
            adj[hit[0]].add(hit[1])
            adj[hit[1]].add(hit[0])
    comps, seen = [], set()
    for f in sorted(crossed):
        if f in seen:
            continue
        stack, comp = [f], set()
        while stack:
            g = stack.pop()
            if g in comp:
                continue
            comp.add(g)
            stack += list(adj[g] - comp)
        seen |= comp
        comps.append(frozenset(comp))
    assert len(comps) > 5
    got = [_face_triples(tr, H, W) for tr in trajs]
    assert sorted(map(frozenset, got), key=sorted) == sorted(comps, key=sorted)
    for path in got:
        assert len(set(path)) == len(path)
        for a, b in zip(path, path[1:]):
            assert b in adj[a]


def test_eps_prime_is_the_largest_safe_integer_bound():
    """R2: fixed-point rounding moves a value by at most 1/2 unit, so a
    reconstruction within eps' units of q stays within eps of x when
    eps' + 1/2 <= eps * 2^k; eps' is the largest such integer (0 when none is
    positive, at most 2^23)."""
    rng = np.random.default_rng(33)
    for _ in range(4000):
        k = int(rng.integers(-10, 40))
        eps = float(rng.uniform(0, 3) * 2.0 ** (-k) * 10.0 ** rng.integers(-1, 3))
        e = oracle.eps_int(eps, k)
        S = Fraction(2) ** k
        limit = Fraction(eps) * S
        assert 0 <= e <= 2 ** 23
        if 0 < e < 2 ** 23:
            assert e + Fraction(1, 2) <= limit < e + Fraction(3, 2)
        elif e == 0:
            assert limit < Fraction(3, 2)
        else:
            assert limit >= 2 ** 23 + Fraction(1, 2)


def test_centre_field():
    H, W, T = 20, 20, 5
    uv = synth.centre_field(H, W, T, 9.4, 10.7)
    q = oracle.to_fixed(uv, oracle.scale_exponent(np.abs(uv).max()))
    m = oracle.face_masks(q)
    assert (_slice_cps(m) == 1).all()
    trajs, pts, bad = oracle.trajectories(q)
    assert bad == 0 and len(trajs) == 1
    slice_pts = [p for f, p in zip(trajs[0], pts[0]) if f % 12 < 2]
    for p in slice_pts:
        assert abs(p[0] - 9.4) < 1e-5 and abs(p[1] - 10.7) < 1e-5


def test_birth_pair_one_trajectory():
    H, W, T = 16, 32, 6
    uv = synth.birth_field(H, W, T, 15.5, 7.5, 6.0, 2)
    q = oracle.to_fixed(uv, oracle.scale_exponent(np.abs(uv).max()))
    cps = _slice_cps(oracle.face_masks(q))
    assert list(cps[:3]) == [0, 0, 0] and (cps[3:] == 2).all()
    trajs, _, bad = oracle.trajectories(q)
    assert bad == 0 and len(trajs) == 1


# ---------------------------------------------------------------------------
# Alg. 2: sufficiency (the bound never lets a non-crossed face become crossed)
# ---------------------------------------------------------------------------
def test_alg2_sufficiency_exhaustive_perturbation():
    rng = np.random.default_rng(11)
    checked = 0
    while checked < 400:
        vals = [int(x) for x in rng.integers(-7, 8, 6)]
        for role in range(3):
            tri = [vals[0:2], vals[2:4], vals[4:6]]
            moved = tri[role]
            others = [tri[r] for r in range(3) if r != role]
            if oracle.face_crossed_batch(np.array(vals))[0]:
                continue
            xi = oracle.alg2(others[0][0], others[0][1], others[1][0], others[1][1], moved[0], moved[1])
            if xi < 1 or xi > 6:
                continue
            for du in range(-xi, xi + 1):
                for dv in range(-xi, xi + 1):
                    t2 = [list(x) for x in tri]
                    t2[role] = [moved[0] + du, moved[1] + dv]
                    assert not oracle.face_crossed_batch(np.array(sum(t2, [])))[0], (vals, role, du, dv)
            checked += 1


def test_alg2_early_returns():
    # M = 0 (collinear values) and a zero neighbour force a lossless vertex
    assert oracle.alg2(1, 1, 2, 2, 3, 3) == 0
    assert oracle.alg2(0, 0, 5, 1, 3, 2) == 0
    assert oracle.alg2(5, 1, 0, 0, 3, 2) == 0
    # all u strictly positive: the bound is at least |u2| - 1
    assert oracle.alg2(4, -3, 6, 5, 9, 1) >= 8


# ---------------------------------------------------------------------------
# Predictors and quantisers
# ---------------------------------------------------------------------------
def test_lorenzo_exact_without_mixed_term():
    """The 3-D Lorenzo prediction error is the mixed third difference, so it is
    exact in the interior for f = g(i,j) + h(i,t) + k(j,t)."""
    rng = np.random.default_rng(3)
    T, H, W = 4, 5, 6
    g = rng.integers(-50, 50, (H, W))
    h = rng.integers(-50, 50, (H, T))
    kk = rng.integers(-50, 50, (W, T))
    Q = np.zeros((T, H, W, 2), np.int32)
    for t in range(T):
        Q[t, :, :, 0] = g + h[:, t][:, None] + kk[:, t][None, :]
        Q[t, :, :, 1] = 3 * g - h[:, t][:, None]
    for t in range(1, T):
        for i in range(1, H):
            for j in range(1, W):
                for c in range(2):
                    assert oracle.lorenzo(Q, t, i, j, c) == Q[t, i, j, c]
    # t = 0 reduces to the 2-D Lorenzo predictor; out-of-domain terms are 0
    assert oracle.lorenzo(Q, 0, 2, 3, 0) == Q[0, 1, 3, 0] + Q[0, 2, 2, 0] - Q[0, 1, 2, 0]
    assert oracle.lorenzo(Q, 0, 0, 0, 0) == 0
    assert oracle.lorenzo(Q, 1, 0, 0, 1) == Q[0, 0, 0, 1]


def _linear_slice(H, W, A, bvec, k):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    u = A[0][0] * x + A[0][1] * y + bvec[0]
    v = A[1][0] * x + A[1][1] * y + bvec[1]
    P = np.stack([u, v], -1) * 2.0 ** k
    assert np.all(P == np.round(P))
    return P.astype(np.int32)


def test_sl_rk2_on_linear_field():
    """Bilinear interpolation reproduces an affine field, so the RK2 departure
    point (Eqs. 7-8) and the sample (Eq. 6) have a closed form."""
    H, W, k = 40, 40, 10
    A = [[0.0, -0.125], [0.125, 0.0]]   # solid-body rotation about (20, 20)
    bvec = [2.5, -2.5]
    P = _linear_slice(H, W, A, bvec, k)
    cfl = 2.0 ** -k
    V = lambda x, y: (A[0][0] * x + A[0][1] * y + bvec[0], A[1][0] * x + A[1][1] * y + bvec[1])
    for i, j in [(20, 20), (15, 25), (24, 12), (18, 30)]:
        u0, v0 = V(j, i)
        assert max(abs(u0), abs(v0)) <= 2.0
        xh, yh = j - 0.5 * u0, i - 0.5 * v0
        uh, vh = V(xh, yh)
        xs, ys = j - uh, i - vh
        pu, pv, mode = oracle.sl_predict(P, i, j, cfl, cfl)
        assert mode == 0
        eu, ev = V(xs, ys)
        assert abs(pu - eu * 2 ** k) <= 1 and abs(pv - ev * 2 ** k) <= 1


def test_sl_substeps_on_linear_field():
    """Above d_max = 2 the departure point is N = ceil(d/2) Euler substeps (Eq. 9)."""
    H, W, k = 64, 64, 8
    A = [[0.0, -0.25], [0.25, 0.0]]
    bvec = [8.0, -8.0]   # rotation about (32, 32), speed 0.25 r
    P = _linear_slice(H, W, A, bvec, k)
    cfl = 2.0 ** -k
    V = lambda x, y: (A[0][0] * x + A[0][1] * y + bvec[0], A[1][0] * x + A[1][1] * y + bvec[1])
    for i, j in [(32, 50), (20, 32), (45, 44)]:
        u0, v0 = V(j, i)
        d = max(abs(u0), abs(v0))
        assert d > 2
        N = min(math.ceil(d / 2), 32)
        x, y = float(j), float(i)
        for _ in range(N):
            us, vs = V(x, y)
            x, y = x - us / N, y - vs / N
        pu, pv, mode = oracle.sl_predict(P, i, j, cfl, cfl)
        assert mode == N
        eu, ev = V(x, y)
        assert abs(pu - eu * 2 ** k) <= 1 and abs(pv - ev * 2 ** k) <= 1


def test_sl_substep_cap():
    H, W, k = 8, 8, 0
    P = np.zeros((H, W, 2), np.int32)
    P[..., 0] = 200   # 200 cells per step: ceil(200/2) > 32
    _, _, mode = oracle.sl_predict(P, 4, 4, 1.0, 1.0)
    assert mode == 32


def test_quantizer_bound():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        xiq = 1 << int(rng.integers(0, 20))
        q = int(rng.integers(-2**23, 2**23))
        p = q + int(rng.integers(-70000 * (2 * xiq + 1), 70000 * (2 * xiq + 1)))
        sym, qh = oracle.quantize(q, p, xiq)
        if sym == 0:
            assert qh == q
        else:
            assert abs(qh - q) <= xiq and qh == p + (sym - 32768) * (2 * xiq + 1)
            assert 0 < sym < 65536


def test_quantizer_bins_are_maximal():
    """With an integer bound xi_q a bin can hold at most 2 xi_q + 1
    consecutive residuals (|r - c w| <= xi_q); the quantiser's bins hold
    exactly that many, tile the residuals in order, and the one around 0 is
    the zero code (r in [-xi_q, xi_q] is reconstructed as the prediction)."""
    for xiq in [1, 2, 4, 64, 1024]:
        p = 12345
        codes = {}
        for r in range(-5 * (2 * xiq + 1), 5 * (2 * xiq + 1)):
            sym, qh = oracle.quantize(p + r, p, xiq)
            assert abs(qh - (p + r)) <= xiq
            codes.setdefault(sym, []).append(r)
        syms = sorted(codes)
        assert syms == list(range(syms[0], syms[-1] + 1))
        for sy in syms[1:-1]:
            rs = codes[sy]
            assert len(rs) == 2 * xiq + 1 and rs == list(range(rs[0], rs[-1] + 1))
        assert codes[32768] == list(range(-xiq, xiq + 1))
        assert oracle.quantize(p + xiq, p, xiq) == (32768, p)


def test_xi_code():
    assert oracle.xi_code(0) == 0
    for x in [1, 2, 3, 4, 7, 8, 1000, 2**23]:
        assert oracle.xi_code(x) == x.bit_length()


def test_fixed_point_scale():
    # R1: the largest magnitude lands in [2^22, 2^23) after scaling by 2^k
    for amax in [0.75, 1.0, 0.5, 3.0, 1e-3, 6.1e4, 2.0**-30]:
        k = oracle.scale_exponent(amax)
        assert 2 ** 22 <= amax * 2.0 ** k < 2 ** 23
    assert oracle.scale_exponent(0.0) == 0
    x = np.array([0.3, -0.7, 1e-3, 0.5], np.float32)
    k = oracle.scale_exponent(0.7)
    q = oracle.to_fixed(x, k)
    assert (q == np.rint(x.astype(np.float64) * 2.0 ** k)).all()


# ---------------------------------------------------------------------------
# MoP scoring (Eq. 10): integer log2 and the entropy estimate
# ---------------------------------------------------------------------------
def test_ilog2_q32_against_math():
    xs = [1, 2, 3, 5, 7, 100, 12345, 2**20 + 1, 2**31 - 1, 2**32 - 1]
    rng = np.random.default_rng(2)
    xs += [int(x) for x in rng.integers(1, 2**32 - 1, 500)]
    for x in xs:
        r = oracle.ilog2_q32(x) / 2.0**32
        assert abs(r - math.log2(x)) < 2e-8, x
        assert r <= math.log2(x) + 1e-12


def test_score_matches_entropy():
    rng = np.random.default_rng(4)
    for _ in range(50):
        hist = np.zeros(65536, np.uint32)
        keys = rng.integers(32768 - 20, 32768 + 20, int(rng.integers(1, 128)))
        for kk in keys:
            hist[kk] += 1
        n = int(hist.sum())
        L = int(rng.integers(0, 10))
        p = hist[hist > 0] / n
        H0 = float(-(p * np.log2(p)).sum())
        want = H0 + 16.0 * L / (n + L) + 1.0 / (2 * 16 * 16)
        got = oracle.score_q32(hist, n, L, 16) / 2.0**32
        assert abs(got - want) < 1e-6


# ---------------------------------------------------------------------------
# MoP block choice (Sec. VI-B) on fields where one predictor is exact
# ---------------------------------------------------------------------------
def _pattern_field(T, H, W, shift, a=0.02):
    """u = 1 + a h(x - shift t, y), v = a g(x - shift t, y): a smooth pattern
    (wavelengths 6 and 7 cells) carried in x by `shift` cells per step; the
    flow itself moves one cell per step in x (|u - 1| <= a)."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    uv = np.empty((T, H, W, 2), np.float32)
    for t in range(T):
        xs = x - shift * t
        h = np.sin(2 * np.pi * xs / 6 + 0.3) * np.cos(2 * np.pi * y / 7 + 1.1)
        g = np.cos(2 * np.pi * xs / 6 - 0.7) * np.sin(2 * np.pi * y / 7 + 0.4)
        uv[t, :, :, 0] = 1.0 + a * h
        uv[t, :, :, 1] = a * g
    return uv


def _interior_modes(res, B=16):
    m = res["modes"]
    return m[1:, 1:-1, 1:-1]


def test_mop_prefers_sl_when_the_flow_carries_the_field():
    """A pattern moved one cell per step by a flow of speed 1: the RK2
    departure point (Eqs. 7-8) of an interior vertex is the vertex one cell
    upstream up to a*|h| <= 0.02 cells, so SL misses by at most that offset
    times the pattern's slope (a * 2 pi / 6) plus the bilinear error, about
    eps = 1e-3 * range in the worst case and a twentieth of it typically,
    while the 3-D Lorenzo error is the pattern's mixed third difference,
    several eps.  Every interior block of every slice t >= 1 must pick SL."""
    uv = _pattern_field(4, 64, 80, shift=1.0)
    res = oracle.compress(uv, 1e-3, pred="mop", block=16)
    assert (res["modes"][0] == 0).all()  # slice 0 has no slice t-1
    assert (_interior_modes(res) == 1).all()
    # the premise, on the fixed-point field
    q, e, k = res["q"], res["stats"]["eps_int"], res["stats"]["k"]
    c = oracle.cfl(1.0, 1.0, k)
    sl_err, lz_err = [], []
    for t in (1, 3):
        for i in range(17, 47, 3):
            for j in range(17, 63, 3):
                pu, pv, mode = oracle.sl_predict(q[t - 1], i, j, c, c)
                assert mode == 0
                sl_err += [abs(pu - q[t, i, j, 0]), abs(pv - q[t, i, j, 1])]
                lz_err += [abs(oracle.lorenzo(q, t, i, j, ch) - q[t, i, j, ch]) for ch in (0, 1)]
    assert max(sl_err) < e / 2 and np.median(sl_err) < e / 8
    assert np.median(lz_err) > 2 * e and min(lz_err) > max(sl_err)


def test_mop_prefers_3dl_on_a_static_field():
    """The same pattern held still: every 3-D Lorenzo term of slice t-1
    cancels its slice-t partner up to the reconstruction error, while SL still
    traces one cell upstream and misses by the pattern's one-cell change
    (about 20 eps).  Every block must keep 3DL."""
    uv = _pattern_field(4, 64, 80, shift=0.0)
    res = oracle.compress(uv, 1e-3, pred="mop", block=16)
    assert (res["modes"] == 0).all()


def test_mop_tie_keeps_3dl():
    """A uniform flow: both predictors are exact, the scores are equal and the
    switching margin (SL must be 0.3 % cheaper) keeps 3DL in every block."""
    uv = np.zeros((3, 40, 48, 2), np.float32)
    uv[..., 0], uv[..., 1] = 0.75, -0.5
    res = oracle.compress(uv, 1e-3, pred="mop", block=16)
    assert (res["modes"] == 0).all()
    assert res["stats"]["sl_blocks"] == 0


def test_time_constant_field_is_lossless():
    """Alg. 2 returns 0 on a face whose values make M = 0.  In a field that
    does not change in time the edge from (t, i, j) to (t + 1, i, j) joins
    equal values, so every face through it is degenerate, and every vertex
    lies on such an edge: Alg. 4 gives xi = 0 everywhere and the whole field
    is stored verbatim (while no face is crossed)."""
    uv = _pattern_field(3, 20, 24, shift=0.0)
    res = oracle.compress(uv, 1e-3, pred="lorenzo")
    assert res["stats"]["crossed_faces"] == 0
    assert (res["xi"] == 0).all() and res["stats"]["lossless_vertices"] == 3 * 20 * 24
    assert (res["qhat"] == res["q"]).all()
    # one step of change in time breaks the degeneracy of the interior vertices
    uv[1:, :, :, 0] += np.float32(0.001) * np.arange(1, 3, dtype=np.float32)[:, None, None]
    uv[1:, :, :, 1] -= np.float32(0.0007) * np.arange(1, 3, dtype=np.float32)[:, None, None]
    assert (oracle.compress(uv, 1e-3, pred="lorenzo")["xi"][:, 2:-2, 2:-2] > 0).any()


# ---------------------------------------------------------------------------
# Canonical length-limited Huffman (package-merge)
# ---------------------------------------------------------------------------
def _huffman_cost(freq):
    h = [int(f) for f in freq if f > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_huffman_optimal_and_complete():
    rng = np.random.default_rng(9)
    for n in [2, 3, 5, 33, 300, 5000]:
        f = rng.integers(0, 1000, n).astype(np.uint64)
        f[rng.integers(0, n)] += 1
        L = oracle.huff_lengths(f)
        used = f > 0
        if used.sum() >= 2:
            assert abs(sum(2.0 ** -int(l) for l in L[used]) - 1.0) < 1e-12
        assert int((L.astype(np.uint64) * f).sum()) == _huffman_cost(f)
        assert L.max() <= 24 and ((L > 0) == used).all()


def test_huffman_length_limit_is_optimal():
    """Against brute force over all length vectors satisfying Kraft <= 1."""
    rng = np.random.default_rng(10)
    for _ in range(25):
        n = int(rng.integers(2, 7))
        maxlen = int(rng.integers(max(2, math.ceil(math.log2(n))), 5))
        f = (rng.random(n) ** 6 * 1000).astype(np.uint64) + 1
        L = oracle.huff_lengths(f, maxlen)
        best = min(sum(int(a) * int(b) for a, b in zip(ls, f))
                   for ls in itertools.product(range(1, maxlen + 1), repeat=n)
                   if sum(2.0 ** -l for l in ls) <= 1.0)
        assert int((L.astype(np.uint64) * f).sum()) == best
        assert L.max() <= maxlen
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    L = oracle.huff_lengths(np.array(fib, np.uint64))
    assert L.max() == 24 and abs(sum(2.0 ** -int(l) for l in L) - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# End to end: pointwise bound, Thm. 1/2 on the round trip
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pred", ["lorenzo", "sl", "mop"])
def test_roundtrip_invariants_vortex64(pred):
    uv = synth.vortex_sum()
    d = oracle.compress(uv, 1e-2, pred=pred)
    qh, x, k = oracle.decompress(d["bytes"])
    assert (qh == d["qhat"]).all()
    st = d["stats"]
    assert np.abs(x.astype(np.float64) - uv.astype(np.float64)).max() <= st["eps"]
    assert (oracle.face_masks(qh) == d["mask"]).all()
    t0, p0, b0 = oracle.trajectories(d["q"])
    t1, p1, b1 = oracle.trajectories(qh)
    assert b0 == b1 == 0 and len(t0) == len(t1)
    assert all((a == b).all() for a, b in zip(t0, t1))
    # a crossed incident face forces a lossless vertex (Alg. 4)
    assert (d["qhat"][d["qxi"] == 0] == d["q"][d["qxi"] == 0]).all()
    assert len(d["bytes"]) < uv.nbytes / 4


def test_xi_zero_where_face_crossed():
    uv = synth.vortex_sum()
    d = oracle.compress(uv, 1e-2, pred="lorenzo")
    m, xi = d["mask"], d["xi"]
    F = oracle.face_table()
    T, H, W = m.shape
    for t, i, j in zip(*np.nonzero(m)):
        for ty in range(12):
            if m[t, i, j] >> ty & 1:
                for e in F[ty]:
                    assert xi[t + e[0], i + e[1], j + e[2]] == 0


def test_forced_vertices_are_lossless_and_the_stream_decodes():
    """Repair reading R14: a forced vertex is stored losslessly (bound code 0,
    reconstruction = input); forcing none changes no byte; the stream decodes
    to the reconstruction and keeps every face predicate."""
    uv = synth.vortex_sum(30, 34, 4, seed=17)
    base = oracle.compress(uv, 1e-2, pred="mop")
    none = oracle.compress(uv, 1e-2, pred="mop", force=np.zeros((4, 30, 34), bool))
    assert none["bytes"] == base["bytes"]
    force = np.zeros((4, 30, 34), bool)
    force[1, 10:13, 7:9] = True
    force[3, 29, 33] = True
    r = oracle.compress(uv, 1e-2, pred="mop", force=force)
    assert (r["qxi"][force] == 0).all() and (r["xi"][force] == 0).all()
    assert (r["qhat"][force] == r["q"][force]).all()
    assert (r["qhat"][:1] == base["qhat"][:1]).all()  # slices before the first forced vertex unchanged
    qh, _, _ = oracle.decompress(r["bytes"])
    assert (qh == r["qhat"]).all()
    assert (oracle.face_masks(qh) == r["mask"]).all()
