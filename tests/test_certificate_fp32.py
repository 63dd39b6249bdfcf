"""The rounding-error certificate of the FP32 nearest-codevector search, checked
on the CPU with exact arithmetic.

The FP32 search (Alg. 1 "Cell Allocation") evaluates, for every row x and
codevector c_n, centred by mu (x~ = fl(x - mu), c~_n = fl(c_n - mu)), the FMA
chain

    v_n = fma(x~_{L-1}, -2 c~_{n,L-1}, ... fma(x~_0, -2 c~_{n,0}, s0_n) ...),
    s0_n = fl32(||c~_n||^2 - k_n),  k_n = fl32_up(2 (L+2) u ||c~_n||^2),  u = 2^-24,

and claims (the proof in the header of the kernel source)

    v_n - R <= f_n <= v_n + 2 k_n + R,   f_n = ||c~_n||^2 - 2 x~.c~_n,  R = (L+2) u ||x~||^2,

so that, with the codevectors taken in split pairs (2k, 2k + 1), V1 = v_i1 the
minimum and V2 the smallest value outside i1's pair, V2 - V1 > 2R + 2k_pair +
4 eta (g1 + eta) (k_pair the larger k of the pair, eta = u (||x~|| + max ||c~||),
g1 >= ||x~ - c~_i1||) proves that the exact argmin of ||x - c_n|| over the
original FP32 values is a member of that pair; the members' FP32 direct-form
distances then decide when they differ by more than their rounding bound.
These tests emulate that chain with every FMA rounded exactly (integer
arithmetic, round to nearest even), then check the bound against the exact f_n
and, on constructed near-ties, that every row the certificate accepts has the
exact (rational) argmin.  They test the mathematics of the certificate; the GPU
parity tests test the kernel.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

U = Fraction(1, 2 ** 24)


# ------------------------------------------------------------ exact rounding
def _round_to_f32(num: int, exp: int, up: bool = False) -> float:
    """num * 2**exp rounded to float32 (nearest even, or toward +inf)."""
    if num == 0:
        return 0.0
    sign = -1 if num < 0 else 1
    mag = abs(num)
    shift = max(mag.bit_length() - 24, -149 - exp)
    if shift > 0:
        q, r = divmod(mag, 1 << shift)
        if up:
            if r and sign > 0:
                q += 1
        else:
            half = 1 << (shift - 1)
            if r > half or (r == half and q & 1):
                q += 1
        mag, exp = q, exp + shift
    out = sign * math.ldexp(mag, exp)
    if abs(out) > float(np.finfo(np.float32).max):
        return math.copysign(math.inf, out)
    return out


def _parts(x: float):
    """x == m * 2**e with integer m (exact for any float)."""
    m, e = math.frexp(x)
    return int(m * (1 << 53)), e - 53


def fma32(a: float, b: float, c: float) -> float:
    ma, ea = _parts(a)
    mb, eb = _parts(b)
    mc, ec = _parts(c)
    E = min(ea + eb, ec)
    total = ma * mb * (1 << (ea + eb - E)) + mc * (1 << (ec - E))
    return _round_to_f32(total, E)


def f32_of(x: Fraction, up: bool = False) -> float:
    """Fraction rounded to float32 (nearest even, or toward +inf)."""
    if x == 0:
        return 0.0
    # enough integer bits below the leading one for a correct rounding
    k = 80 - (abs(x.numerator).bit_length() - x.denominator.bit_length())
    num = x.numerator * (1 << k) if k >= 0 else x.numerator
    den = x.denominator if k >= 0 else x.denominator * (1 << -k)
    q, r = divmod(abs(num), den)
    # fold the remainder into a sticky bit below the kept bits
    q = (q << 1) | (1 if r else 0)
    return _round_to_f32(q if num > 0 else -q, -k - 1, up=up)


def test_exact_rounding_helpers():
    """fma32 and f32_of against numpy's float32 rounding where a single
    correctly rounded double is exact (so numpy rounds once), including
    halfway cases, and against the definition of rounding up."""
    rng = np.random.default_rng(0)
    for _ in range(3000):
        a, b, c = (float(np.float32(v)) for v in rng.integers(-2 ** 12, 2 ** 12, 3))
        exact = a * b + c          # exact in double: |a b + c| < 2**25
        assert fma32(a, b, c) == float(np.float32(exact))
    # halfway cases: 2**24 + 1 and 2**24 + 3 are ties between float32 neighbours
    assert fma32(1.0, float(2 ** 24), 1.0) == float(2 ** 24)          # tie to even (down)
    assert fma32(1.0, float(2 ** 24), 3.0) == float(2 ** 24 + 4)      # tie to even (up)
    assert fma32(1.0, float(2 ** 24), -1.0) == float(2 ** 24 - 1)     # exact below 2**24
    for _ in range(2000):
        x = Fraction(int(rng.integers(1, 2 ** 40)), int(rng.integers(1, 2 ** 40)))
        d = f32_of(x)
        assert d == float(np.float32(float(x))) or abs(Fraction(d) - x) <= abs(
            Fraction(float(np.float32(float(x)))) - x)
        up = f32_of(x, up=True)
        assert Fraction(up) >= x and float(np.float32(up)) == up
        assert Fraction(float(np.nextafter(np.float32(up), np.float32(0)))) < x


# ------------------------------------------------------- the search's chain
def chain(xt, ct, L):
    """(v_n, k_n) of the FP32 search for one centred row xt against centred
    codevectors ct (lists of float32 values)."""
    out = []
    for c in ct:
        sq = 0.0
        for l in range(L):      # FP64 norm (the preparation kernel's precision)
            sq += c[l] * c[l]
        k = f32_of(Fraction(2 * (L + 2)) * U * Fraction(sq), up=True)
        v = f32_of(Fraction(sq) - Fraction(k))
        for l in range(L):
            v = fma32(xt[l], -2.0 * c[l], v)
        out.append((v, k))
    return out


def centred(X, C, mu):
    xt = [[float(np.float32(x) - np.float32(m)) for x, m in zip(row, mu)] for row in X]
    ct = [[float(np.float32(c) - np.float32(m)) for c, m in zip(row, mu)] for row in C]
    return xt, ct


@pytest.mark.parametrize("L,scale,offset", [(1, 1.0, 0.0), (4, 1e3, 0.0), (16, 255.0, 128.0),
                                            (64, 1.0, 1e4), (128, 1e-3, 0.0)])
def test_chain_error_within_certificate_bound(L, scale, offset):
    """v_n - R <= f_n <= v_n + 2 k_n + R for every (row, codevector), on data
    with a large common offset and a centring vector away from the data
    (strong cancellation in x~.c~), and with codevectors near the rows."""
    rng = np.random.default_rng(L)
    X = (offset + scale * rng.standard_normal((6, L))).astype(np.float32)
    C = np.concatenate([X[:3] + (scale * 1e-3 * rng.standard_normal((3, L))).astype(np.float32),
                        (offset + scale * rng.standard_normal((5, L))).astype(np.float32)])
    mu = (offset * 0.5 + scale * rng.standard_normal(L)).astype(np.float32)
    xt, ct = centred(X, C, mu)
    for x in xt:
        xq = [Fraction(v) for v in x]
        R = (L + 2) * U * sum(v * v for v in xq)
        for (v, k), c in zip(chain(x, ct, L), ct):
            cq = [Fraction(t) for t in c]
            f = sum(t * t for t in cq) - 2 * sum(a * b for a, b in zip(xq, cq))
            assert Fraction(v) - R <= f <= Fraction(v) + 2 * Fraction(k) + R


def _pair_top2(vals):
    """(i1, V1, V2): the minimum, its index (lowest on ties) and the smallest
    value outside i1's split pair (2k, 2k + 1)."""
    i1 = min(range(len(vals)), key=lambda n: (vals[n], n))
    out = [vals[n] for n in range(len(vals)) if n // 2 != i1 // 2]
    return i1, vals[i1], (min(out) if out else Fraction(10) ** 60)


def direct32(x, c):
    """The FP32 direct-form distance sum_l (x_l - c_l)^2 in index order (FMA)."""
    d = 0.0
    for a, b in zip(x, c):
        t = float(np.float32(a) - np.float32(b))
        d = fma32(t, t, d)
    return d


def _resolve(i1, N, dist, L):
    """The member of i1's pair with the smaller direct-form distance when the two
    differ by more than (L + 4) u (da + db); None when they do not."""
    ip = i1 ^ 1
    if ip >= N:
        return i1
    da, db = Fraction(dist(i1)), Fraction(dist(ip))
    tol = (L + 4) * U * (da + db)
    if db < da - tol:
        return ip
    return i1 if da < db - tol else None


def _certify(x_orig, C_orig, mu, L):
    """(certified, chosen index) from the emulated chain and the certificate's
    margin, evaluated in exact arithmetic (the kernel evaluates it in FP32 with
    a 2^-15 relative slack), then the pair resolved by FP32 direct distances."""
    (xt,), ct = centred([x_orig], C_orig, mu)
    vk = chain(xt, ct, L)
    vals = [Fraction(v) for v, _ in vk]
    N = len(vals)
    i1, V1, V2 = _pair_top2(vals)
    xn2 = sum(Fraction(v) ** 2 for v in xt)
    R = (L + 2) * U * xn2
    cmax = max(math.sqrt(sum(t * t for t in c)) for c in ct)
    eta = U * Fraction(math.sqrt(float(xn2)) * (1 + 2 ** -50) + cmax * (1 + 2 ** -50))
    g1 = Fraction(math.sqrt(float(sum((Fraction(a) - Fraction(b)) ** 2
                                      for a, b in zip(xt, ct[i1])))) * (1 + 2 ** -50))
    kp = max(Fraction(vk[n][1]) for n in (i1, i1 ^ 1) if n < N)
    margin = 2 * R + 2 * kp + 4 * eta * (g1 + eta)
    if not V2 - V1 > margin:
        return False, i1
    win = _resolve(i1, N, lambda n: direct32(x_orig, C_orig[n]), L)
    return (win is not None), (i1 if win is None else win)


@pytest.mark.parametrize("family", ["pair_near_row", "pair_far_row_at_mu", "mu_far_from_row"])
def test_certified_rows_are_exact_on_near_ties(family):
    """Rows equidistant (up to float32 rounding) from two codevectors, moved
    apart by eps from 0 up: the certificate must accept only rows whose exact
    argmin it names, and both outcomes must occur.  The three families put the
    rounding error where each term of the margin covers it: codevectors near
    the row (all terms small), a far pair with the row at the centring vector
    (the chain start's rounding, covered by k), and a centring vector far from
    row and codevectors (the cross term's cancellation, covered by R)."""
    rng = np.random.default_rng({"pair_near_row": 7, "pair_far_row_at_mu": 9,
                                 "mu_far_from_row": 11}[family])
    L = 8
    spread = {"pair_near_row": 20.0, "pair_far_row_at_mu": 1000.0, "mu_far_from_row": 20.0}[family]
    accepted = refused = 0
    for trial in range(300):
        x = (128 + 40 * rng.standard_normal(L)).astype(np.float32)
        c0 = (x + spread * rng.standard_normal(L)).astype(np.float32)
        # c1: c0 reflected across a hyperplane through x (equidistant up to
        # rounding), then moved by eps in a random direction
        w = rng.standard_normal(L)
        w /= np.linalg.norm(w)
        d = c0.astype(np.float64) - x
        c1 = x + d - 2 * np.dot(d, w) * w
        eps = 0.0 if trial % 4 == 0 else spread * 10 ** rng.uniform(-9, 0)
        v = rng.standard_normal(L)
        c1 = (c1 + eps * v / np.linalg.norm(v)).astype(np.float32)
        far = (x + 10 * spread + 50 * rng.standard_normal((3, L))).astype(np.float32)
        C = np.concatenate([[c0], [c1], far]) if trial % 3 else np.concatenate([[c1], far, [c0]])
        if family == "pair_near_row":
            mu = C.mean(0, dtype=np.float32)
        elif family == "pair_far_row_at_mu":
            mu = (x + 1e-3 * rng.standard_normal(L)).astype(np.float32)
        else:
            mu = (x - 2000 + 100 * rng.standard_normal(L)).astype(np.float32)
        ok, i1 = _certify(x, C, mu, L)
        exact = [sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, c))
                 for c in C]
        best = min(range(len(C)), key=lambda n: (exact[n], n))
        if ok:
            accepted += 1
            assert i1 == best, f"trial {trial}: certified {i1}, exact argmin {best}"
            assert exact[i1] < min(e for n, e in enumerate(exact) if n != i1)
        else:
            refused += 1
    assert accepted > 0 and refused > 0


def _worst_case_margin_check(x, C, mu, L, weights=(1, 1, 1)):
    """Worst case allowed by the bound: every v_n anywhere in
    [f_n - 2k_n - R, f_n + R].  The adversary pushes the exact winner b up and
    every other codevector down.  Returns "refused", "right" (accepted, names
    the exact argmin) or "wrong" (accepted another codevector).  `weights`
    scale the margin's three terms (2R, 2k, the eta term) to show that each is
    needed."""
    (xt,), ct = centred([x], C, mu)
    xq = [Fraction(v) for v in xt]
    xn2 = sum(v * v for v in xq)
    R = (L + 2) * U * xn2
    exact = [sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, c)) for c in C]
    b = min(range(len(C)), key=lambda n: (exact[n], n))
    v = []
    for n, c in enumerate(ct):
        cq = [Fraction(t) for t in c]
        sq = sum(t * t for t in cq)
        k = Fraction(f32_of(2 * (L + 2) * U * sq, up=True))
        f = sq - 2 * sum(a * t for a, t in zip(xq, cq))
        v.append((f + R, k) if n == b else (f - 2 * k - R, k))
    N = len(v)
    i1, V1, V2 = _pair_top2([t[0] for t in v])
    cmax = max(math.sqrt(sum(t * t for t in c)) for c in ct)
    eta = U * Fraction(math.sqrt(float(xn2)) * (1 + 2 ** -50) + cmax * (1 + 2 ** -50))
    g1 = Fraction(math.sqrt(float(sum((a - Fraction(t)) ** 2 for a, t in zip(xq, ct[i1]))))
                  * (1 + 2 ** -50))
    wR, wk, we = (Fraction(w) for w in weights)
    kp = max(v[n][1] for n in (i1, i1 ^ 1) if n < N)
    margin = wR * 2 * R + wk * 2 * kp + we * 4 * eta * (g1 + eta)
    if V2 - V1 > margin:
        # the pair's direct-form distances at the worst end of their rounding bound
        win = _resolve(i1, N, lambda n: exact[n] * (1 + (L + 2) * U if n == b else 1 - (L + 2) * U), L)
        if win is None:
            return "refused"
        ok = win == b and exact[b] < min(e for n, e in enumerate(exact) if n != b)
        return "right" if ok else "wrong"
    return "refused"


FAMILIES = ["pair_near_row", "pair_far_row_at_mu", "mu_far_from_row"]


def _near_tie_rows(family, trials=300):
    """Near-tie pairs: c0 around the row, c1 its reflection across a hyperplane
    through the row moved by eps, three farther codevectors; mu by family."""
    rng = np.random.default_rng(3)
    L = 8
    spread = {"pair_near_row": 20.0, "pair_far_row_at_mu": 1000.0, "mu_far_from_row": 20.0}[family]
    for trial in range(trials):
        x = (128 + 40 * rng.standard_normal(L)).astype(np.float32)
        c0 = (x + spread * rng.standard_normal(L)).astype(np.float32)
        w = rng.standard_normal(L)
        w /= np.linalg.norm(w)
        d = c0.astype(np.float64) - x
        c1 = x + d - 2 * np.dot(d, w) * w
        eps = 0.0 if trial % 4 == 0 else spread * 10 ** rng.uniform(-9, 0)
        v = rng.standard_normal(L)
        c1 = (c1 + eps * v / np.linalg.norm(v)).astype(np.float32)
        far = (x + 10 * spread + 5 * spread * rng.standard_normal((3, L))).astype(np.float32)
        C = np.concatenate([[c0], [c1], far]) if trial % 3 else np.concatenate([[c1], far, [c0]])
        if family == "pair_near_row":
            mu = C.mean(0, dtype=np.float32)
        elif family == "pair_far_row_at_mu":
            mu = (x + 1e-3 * rng.standard_normal(L)).astype(np.float32)
        else:
            mu = (x - 2000 + 100 * rng.standard_normal(L)).astype(np.float32)
        yield x, C, mu, L


@pytest.mark.parametrize("family", FAMILIES)
def test_certificate_sound_at_the_bound(family):
    """Near-tie pairs as above, with every computed value at the worst end of
    the proven interval: no wrong row may be accepted, and rows with a clear
    enough gap still are."""
    outcomes = [_worst_case_margin_check(x, C, mu, L) for x, C, mu, L in _near_tie_rows(family)]
    assert "wrong" not in outcomes
    assert "right" in outcomes


@pytest.mark.parametrize("weights", [(0, 1, 1), (1, 0, 1), (1, 1, 0), (0.5, 1, 1), (1, 0.5, 1)])
def test_each_margin_term_is_needed(weights):
    """Unlike random rounding, the adversary above uses the whole error budget:
    a margin without one of its terms (2R, 2k, the eta term), or with 2R or 2k
    halved, accepts a wrong row in one of the families.  (The eta term covers
    the difference between the centred and the original order; on the exact
    reflections of eps = 0 the two disagree.)"""
    for family in FAMILIES:
        for x, C, mu, L in _near_tie_rows(family):
            if _worst_case_margin_check(x, C, mu, L, weights) == "wrong":
                return
    pytest.fail(f"margin weights {weights}: no wrong row accepted")


def test_certificate_accepts_clear_winners():
    """Away from ties the certificate holds: a row next to one codevector of a
    spread codebook is always accepted (the exact fallback is for near-ties)."""
    rng = np.random.default_rng(8)
    L = 16
    C = (128 + 60 * rng.standard_normal((16, L))).astype(np.float32)
    mu = C.mean(0, dtype=np.float32)
    for n in range(16):
        x = (C[n] + rng.standard_normal(L)).astype(np.float32)
        ok, i1 = _certify(x, C, mu, L)
        assert ok and i1 == n


def test_certificate_resolves_split_twins():
    """Right after a split every codevector has a twin at 2 delta (children 2i, 2i + 1).
    A row near one parent has the two twins as its nearest codevectors; they share a pair,
    so the bound is taken against the next parent and the twins are told apart by their
    exact distances: the row is certified with its exact nearest twin."""
    rng = np.random.default_rng(12)
    L = 16
    parents = (128 + 50 * rng.standard_normal((8, L))).astype(np.float32)
    C = np.empty((16, L), np.float32)
    C[0::2] = parents + np.float32(0.01)
    C[1::2] = parents - np.float32(0.01)
    mu = C.mean(0, dtype=np.float32)
    accepted = 0
    for n in range(8):
        for _ in range(3):
            x = (parents[n] + 2 * rng.standard_normal(L)).astype(np.float32)
            ok, i1 = _certify(x, C, mu, L)
            exact = [sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, c)) for c in C]
            best = min(range(16), key=lambda k: (exact[k], k))
            if ok:
                accepted += 1
                assert i1 == best and best // 2 == n
    assert accepted >= 20
