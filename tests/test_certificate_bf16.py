"""The two certificates of the BF16 tensor-core nearest-codevector search,
checked on the CPU under the library's accumulation model.

The tensor-core search (Alg. 1 "Cell Allocation" with the cross term on
tcgen05 MMAs) works with an integer centring vector mu, integer rows
x~ = x - mu (8-bit image samples), and codevectors c~ = fl32(c - mu) whose
scaled value c' = -2 c~ is split into two BF16 pieces p_hi + p_mid with the
exact remainder r = c' - p_hi - p_mid.  One MMA row accumulates

    G_n = X2 + s0_n + x~ . (p_hi + p_mid),   X2 = ||x~||^2,
    s0_n = fl32(||c~||^2 - k'_n),  k'_n = fl32_up((2 tau + 2^-23) ||c~||^2),

and the library assumes the FP32 accumulation error stays within
tau * (sum_l |x~_l c'_l| + |s0_n| + X2), tau = (K/16 + 2) 2^-22 (1 + 2^-7),
K = 2 ceil16(L) + 16.  These tests take that model at its worst: the
accumulator value of the exact winner is pushed to the top of its interval
and every other value to the bottom.  The epilogue is then emulated in FP32
as the kernel runs it (groups of eight columns, the group index packed into
the low mantissa bits of the group minimum, running top-2 of group minima per
chain, merges), the eight members of the best group get FP32 direct
distances at the worst end of their rounding bound, the winner among them
must beat the others by the rounding bound, and both certificates are
evaluated in exact arithmetic.  A row either of them accepts must have the
exact (rational) argmin of the original FP32 values.  This checks the
algebra of the certificates under the model; the measured accumulation
error behind the model, and the kernel itself, are checked on the GPU.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

U = Fraction(1, 2 ** 24)
NT, HALF = 144, 72                  # codevectors per tile, per half
# group size -> bits of the in-half group index; packing moves a group minimum by less than
# 2^(JBITS - 23) of it (at most 2^JBITS - 1 units in the last place)
JBITS = {2: 6, 4: 5, 8: 4}


def round_bits(x: Fraction, p: int, up: bool = False) -> Fraction:
    """x rounded to p significant bits (nearest even, or toward +inf)."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    unit = Fraction(2) ** (e - p + 1)
    q, r = divmod(a, unit)
    q = int(q)
    if up:
        if r and x > 0:
            q += 1
        if r and x < 0:
            pass
    else:
        half = unit / 2
        if r > half or (r == half and q & 1):
            q += 1
    return (q * unit) if x > 0 else -(q * unit)


def f32(x: Fraction, up: bool = False) -> Fraction:
    return round_bits(Fraction(x), 24, up)


def bf16(x: Fraction) -> Fraction:
    return round_bits(Fraction(x), 8)


def sqrt_up(x: Fraction) -> Fraction:
    return Fraction(math.sqrt(float(x)) * (1 + 2 ** -50)) if x > 0 else Fraction(0)


def test_rounding_helpers():
    assert f32(Fraction(2 ** 24 + 1)) == 2 ** 24
    assert f32(Fraction(2 ** 24 + 3)) == 2 ** 24 + 4
    assert f32(Fraction(2 ** 24 + 1), up=True) == 2 ** 24 + 2
    assert bf16(Fraction(257)) == 256 and bf16(Fraction(259)) == 260
    rng = np.random.default_rng(0)
    vals = rng.standard_normal(500) * 10.0 ** rng.integers(-6, 6, 500)
    for v in vals:
        assert f32(Fraction(float(v))) == Fraction(float(np.float32(v)))
    v32 = vals.astype(np.float32)
    for a, b in zip(v32, bf16_rne(v32)):
        assert Fraction(float(b)) == bf16(Fraction(float(a)))
    ties = np.array([257.0, 259.0, -257.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], np.float32)
    np.testing.assert_array_equal(bf16_rne(ties), [256.0, 260.0, -256.0, 1.0, 1.0 + 2.0 ** -6])


def _f32bits_key(lo: np.float32, j: int, jbits: int) -> np.float32:
    b = np.array([lo], np.float32).view(np.uint32)
    b = (b & np.uint32(~((1 << jbits) - 1) & 0xFFFFFFFF)) | np.uint32(j)
    return b.view(np.float32)[0]


def _epilogue(v, GRP):
    """Top-2 of the kernel's epilogue over one row's FP32 accumulator values v
    (length a multiple of NT), groups of GRP columns: (V1, V2, i1), V1 the
    smallest value, V2 the smallest outside V1's group, i1 the first column of
    V1's group."""
    nt = len(v) // NT
    halves = []
    for h in range(2):
        c1, c2, cg = [np.float32(np.inf)] * 2, [np.float32(np.inf)] * 2, [0, 0]
        for t in range(nt):
            s1 = list(c1)
            keys = []
            for j in range(HALF // GRP):
                base = t * NT + h * HALF + GRP * j
                lo = np.float32(min(v[base:base + GRP]))
                keys.append(_f32bits_key(lo, j, JBITS[GRP]))
            # groups enter two at a time, pair p into chain p % 2 (an odd last one alone)
            for p in range(0, len(keys) - 1, 2):
                q = (p // 2) % 2
                m, hh = min(keys[p], keys[p + 1]), max(keys[p], keys[p + 1])
                c2[q] = min(c2[q], max(c1[q], m), hh)
                c1[q] = min(c1[q], m)
            if len(keys) % 2:
                q, k = (len(keys) // 2) % 2, keys[-1]
                c2[q] = min(c2[q], max(c1[q], k))
                c1[q] = min(c1[q], k)
            for q in range(2):
                if c1[q] < s1[q]:
                    cg[q] = t
        jm = (1 << JBITS[GRP]) - 1
        V1, V2 = c1[0], c2[0]
        i1 = cg[0] * NT + h * HALF + GRP * (int(np.array([c1[0]]).view(np.uint32)[0]) & jm)
        iq = cg[1] * NT + h * HALF + GRP * (int(np.array([c1[1]]).view(np.uint32)[0]) & jm)
        V2 = min(min(V2, c2[1]), max(V1, c1[1]))
        if c1[1] < V1 or (c1[1] == V1 and iq < i1):
            V1, i1 = c1[1], iq
        halves.append((V1, V2, i1))
    (A1, A2, ai), (B1, B2, bi) = halves
    V2 = min(min(A2, B2), max(A1, B1))
    if B1 < A1 or (B1 == A1 and bi < ai):
        return B1, V2, bi
    return A1, V2, ai


def bf16_rne(a):
    """float32 array rounded to BF16 (nearest even), returned as float32."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _ints(arrays):
    """Exact integer images of float arrays under one common scale:
    (list of object arrays of Python ints, S) with a == ints * 2**-S."""
    S = 0
    for a in arrays:
        f = np.asarray(a, np.float64)
        nz = f[f != 0]
        if nz.size:
            S = max(S, int(53 - np.frexp(nz)[1].min()))
    out = []
    for a in arrays:
        f = np.asarray(a, np.float64) * 2.0 ** S
        out.append(np.array([int(v) for v in f.ravel()], dtype=object).reshape(f.shape))
    return out, S


def _epilogue_worst(v, best, GRP):
    """The epilogue's top-2 of group minima in exact arithmetic with its one
    rounding effect at its worst: a group minimum moved by its packing (at most
    2^JBITS - 1 units in the last place of an FP32 value, < 2^(JBITS - 23) of
    it), up for the exact winner's group and down for every other group.
    Returns (V1, V2, i1)."""
    c1 = c2 = None
    i1 = -1
    for g in range(len(v) // GRP):
        lo = min(v[GRP * g:GRP * g + GRP])
        s = 1 if GRP * g <= best < GRP * g + GRP else -1
        k = lo + s * Fraction((1 << JBITS[GRP]) - 1, 2 ** 23) * abs(lo)
        if c1 is None:
            c1, c2, i1 = k, Fraction(10) ** 40, GRP * g
            continue
        c2 = min(c2, max(c1, k))
        if k < c1:
            c1, i1 = k, GRP * g
    return c1, c2, i1


def tau_model(Lk):
    """The accumulation-error coefficient the library assumes, (K/16 + 2) 2^-22
    (1 + 2^-7) of (sum |products| + |s0| + X2), with K = 3 Lk + 16 accumulated
    elements for Lk <= 32 (the split form's x_lo . p_hi included), 2 Lk + 16
    otherwise."""
    K = 3 * Lk + 16 if Lk <= 32 else 2 * Lk + 16
    return Fraction(K // 16 + 2, 2 ** 22) * Fraction(129, 128)


def tau_of(Lk):
    """The coefficient of the kernel's margins (k', R'): the model's, times
    1 + 2^-6 for Lk <= 32, where the split form's products may exceed
    ||x~||^2 + ||c~||^2 by 2^-7 of it."""
    return tau_model(Lk) * (Fraction(65, 64) if Lk <= 32 else 1)


def certify(x, C, mu, N, adversarial=True, worst=False, weights=None, GRP=2):
    """Run one row through the model and the two certificates.  With
    worst=True every bounded quantity is at the end of its bound that favours
    a wrong answer (see test_bf16_certificates_sound_at_every_bound).
    `weights` (keys m_R, m_k, m_pack, m_E, lb_R, lb_E, lb_pack) scale terms of
    the first certificate's margin and of the second one's lower bound, to show
    that each is needed.  Rows whose centred values are not integers take the
    split form (x~ = x_hi + x_lo + rem in BF16 pieces; only Lk <= 32).
    Returns (accepted, chosen index, exact argmin)."""
    wt = {k: Fraction(1) for k in ("m_R", "m_k", "m_pack", "m_E", "lb_R", "lb_E", "lb_pack")}
    wt.update({k: Fraction(v) for k, v in (weights or {}).items()})
    L = len(x)
    Lk = -(-L // 16) * 16
    tau = tau_of(Lk)
    taum = tau_model(Lk)
    x = np.asarray(x, np.float32)
    C = np.asarray(C, np.float32)
    mu = np.asarray(mu, np.float32)
    xt32 = (x - mu).astype(np.float32)             # x~ = fl32(x - mu), as the kernel forms it
    split = not np.all(xt32 == np.rint(xt32))
    assert not split or Lk <= 32
    xh = bf16_rne(xt32)
    xl = bf16_rne((xt32 - xh).astype(np.float32))   # x~ - x_hi is exact in FP32
    # exact squared distances of the original FP32 values
    (xi, ci), Sd = _ints([x, C])
    diff = ci - xi[None, :]
    exact = [Fraction(int(v), 1 << (2 * Sd)) for v in (diff * diff).sum(1)]
    best = min(range(N), key=lambda n: (exact[n], n))
    # operands: c~ = fl32(c - mu), c' = -2 c~ = p_hi + p_mid + r (each step exact in FP32)
    ct = (C - mu[None, :]).astype(np.float32)
    cp = (np.float32(-2.0) * ct).astype(np.float32)
    ph = bf16_rne(cp)
    r1 = (cp - ph).astype(np.float32)
    pm = bf16_rne(r1)
    r = (r1 - pm).astype(np.float32)
    (cti, cpi, phi, pmi, ri, r1i, xti, xhi, xli), S = _ints([ct, cp, ph, pm, r, r1, xt32, xh, xl])
    assert np.all(cpi == phi + r1i) and np.all(r1i == pmi + ri)
    sq_exact = [Fraction(int(v), 1 << (2 * S)) for v in (cti * cti).sum(1)]
    scale = 1 << S
    xn2 = Fraction(int((xti * xti).sum()), scale * scale)        # ||x~||^2
    if split:
        # X2 as the kernel forms it: sum (x_hi + x_lo)^2 in FP32, at the top of its bound in
        # the worst case
        # (|fl(sum (x_hi + x_lo)^2) - ||x~||^2| <= ((L + 2) u + 2^-14) ||x~||^2)
        hl = xhi + xli
        X2 = Fraction(int((hl * hl).sum()), scale * scale)
        X2 = xn2 * (1 + (L + 2) * U + Fraction(1, 2 ** 14)) if worst else Fraction(f32(X2))
    else:
        X2 = xn2
        assert X2 < 2 ** 24          # exact in FP32 for these data
    # k'_n rounded up and s0_n rounded to nearest from the FP64 norm, as the preparation does
    s0 = np.empty(N, np.float32)
    kp = []
    for n in range(N):
        sq = float(sq_exact[n])
        k64 = (2.0 * float(tau) + 2.0 ** -23) * sq
        kf = np.float32(k64)
        if float(kf) < k64:
            kf = np.nextafter(kf, np.float32(np.inf))
        kp.append(Fraction(float(kf)))
        s0[n] = np.float32(sq - float(kf))
    (s0i,), S0 = _ints([s0])
    sc2 = scale * scale
    # what the MMAs sum: x_hi . (p_hi + p_mid) (+ x_lo . p_hi on a split row)
    dot = (phi + pmi) @ xhi + (phi @ xli if split else 0)
    adot = (np.abs(phi) + np.abs(pmi)) @ np.abs(xhi) + (np.abs(phi) @ np.abs(xli) if split else 0)
    rnorm = [sqrt_up(Fraction(int(v), sc2)) for v in (ri * ri).sum(1)]
    rho = max(rnorm)
    cmax = max(sqrt_up(q) for q in sq_exact)
    if split:   # the terms the pieces miss, as the kernel bounds them
        E = sqrt_up(xn2) * (rho + Fraction(1, 2 ** 14) * cmax) * Fraction(129, 128)
    else:
        E = sqrt_up(xn2) * rho
    dotc = cpi @ xti                               # x~ . c'
    v = []
    for n in range(N):
        s0n = Fraction(int(s0i[n]), 1 << S0)
        up = (n == best) == adversarial
        if worst:   # the missed terms anywhere in [-E, E]
            G = X2 + s0n + Fraction(int(dotc[n]), sc2) + (E if up else -E)
        else:
            G = X2 + s0n + Fraction(int(dot[n]), sc2)
        Sn = Fraction(int(adot[n]), sc2) + abs(s0n) + X2
        e = taum * Sn if up else -taum * Sn
        if worst:
            v.append(G + e)
            continue
        target = G + e
        # an FP32 value inside the model's interval: round toward G
        val = f32(target, up=True) if e < 0 else -f32(-target, up=True)
        v.append(np.float32(float(val)))
    if worst:
        v += [Fraction(2) ** 100] * (-(-N // GRP) * GRP - N)
        V1, V2, i1 = _epilogue_worst(v, best, GRP)
    else:
        npad = -(-N // NT) * NT
        v += [np.float32(2.0 ** 100)] * (npad - N)
        V1, V2, i1 = _epilogue(v, GRP)
        V1, V2 = Fraction(float(V1)), Fraction(float(V2))

    # FP32 direct-form distances of the group, at the worst end of their bound
    def direct(n):
        d = exact[n]
        return d * (1 + (L + 2) * U) if (n == best) == adversarial else d * (1 - (L + 2) * U)

    members = [n for n in range(i1, i1 + GRP) if n < N]
    dd = {n: direct(n) for n in members}
    ii = min(members, key=lambda n: (dd[n], n))
    da = dd[ii]
    for n in members:
        if n != ii and not (da < dd[n] - (L + 4) * U * (da + dd[n])):
            return False, ii, best
    ka = max(kp[n] for n in members)        # k' of V1's member is only known to be <= this
    R = 2 * tau * X2
    eta = U * (sqrt_up(Fraction(X2)) + cmax)
    pack = Fraction(1, 2 ** (23 - JBITS[GRP])) * (abs(V1) + abs(V2))
    xerr = (L + 2) * U * X2 + (Fraction(1, 2 ** 14) * X2 if split else 0)
    g1 = sqrt_up(V1 + 2 * ka + R + pack + E + xerr)
    margin = (wt["m_R"] * 2 * R + wt["m_k"] * 2 * ka + wt["m_pack"] * pack + wt["m_E"] * 2 * E
              + 4 * eta * (g1 + eta))
    if V2 - V1 > margin:
        return True, ii, best
    lb = V2 - (wt["lb_R"] * R + wt["lb_E"] * E + wt["lb_pack"] * pack + xerr)
    ub = da * (1 + (L + 4) * U)
    if lb > 0 and lb - 2 * eta * sqrt_up(lb) > ub:
        return True, ii, best
    return False, ii, best


def _rows(rng, L, N, spread, trials, family="near"):
    """Integer rows, and codebooks holding a near-tie pair for each row: c0
    near the row ("near"; mu = the rounded codebook mean) or near 2 mu - x
    ("mirror"; mu = the row moved by up to 40 per component, so that
    c~0 = -x~ and the bound sum |x~ c'| <= ||x~||^2 + ||c~||^2 behind the
    accumulation error is tight), c1 its reflection across a hyperplane through
    the row moved by eps (0 in a quarter of the cases), placed in the same
    column pair, in different pairs of one half, or in different halves."""
    for trial in range(trials):
        x = rng.integers(0, 256, L).astype(np.float32)
        if family == "mirror":
            mu = (x + rng.integers(-40, 41, L)).astype(np.float32)
            c0 = (2 * mu - x + spread * rng.standard_normal(L)).astype(np.float32)
        else:
            c0 = (x + spread * rng.standard_normal(L)).astype(np.float32)
        w = rng.standard_normal(L)
        w /= np.linalg.norm(w)
        d = c0.astype(np.float64) - x
        c1 = x + d - 2 * np.dot(d, w) * w
        eps = 0.0 if trial % 4 == 0 else spread * 10 ** rng.uniform(-7, 0)
        dv = rng.standard_normal(L)
        c1 = (c1 + eps * dv / np.linalg.norm(dv)).astype(np.float32)
        if family == "mirror":
            r0 = float(np.linalg.norm(d))
            C = (x + 2 * r0 / np.sqrt(L) * rng.choice([-1, 1], (N, L))
                 + rng.standard_normal((N, L))).astype(np.float32)
        else:
            C = (x + spread * (2.5 + rng.standard_normal((N, L)))).astype(np.float32)
        where = trial % 3
        p0 = 2 * int(rng.integers(0, N // 2))
        p1 = {0: p0 + 1, 1: (p0 + 6) % N, 2: (p0 + HALF + 3) % N}[where]
        C[p0], C[p1] = (c0, c1) if trial % 2 else (c1, c0)
        if family != "mirror":
            mu = np.rint(C.mean(0)).astype(np.float32)
        yield x, C, mu


@pytest.mark.parametrize("GRP", [2, 4, 8])
@pytest.mark.parametrize("L,spread,family", [(16, 20.0, "near"), (16, 2.0, "near"),
                                              (64, 20.0, "near"), (64, 2.0, "near"),
                                              (16, 0.5, "mirror"), (64, 0.5, "mirror")])
def test_bf16_certificates_sound_at_the_model_bound(L, spread, family, GRP):
    rng = np.random.default_rng(L + int(spread))
    N = NT
    trials = 60 if L == 64 else 120
    accepted = 0
    for x, C, mu in _rows(rng, L, N, spread, trials, family):
        ok, ii, best = certify(x, C, mu, N, GRP=GRP)
        if ok:
            accepted += 1
            assert ii == best, (ii, best)
    assert accepted > 0


@pytest.mark.parametrize("GRP", [2, 4, 8])
@pytest.mark.parametrize("L,spread,family", [(16, 20.0, "near"), (16, 2.0, "near"),
                                              (64, 20.0, "near"), (64, 2.0, "near"),
                                              (16, 0.5, "mirror"), (64, 0.5, "mirror")])
def test_bf16_certificates_sound_at_every_bound(L, spread, family, GRP):
    """The proof uses each error only through its bound, so it must hold with
    every error at the end of its bound that favours a wrong answer: the
    accumulation error (model), the missed term x~.r_n anywhere in
    [-||x~|| rho, ||x~|| rho], the packed group minimum and the direct-form
    distances of the group's members.  With all of them at
    their worst, no wrong row is accepted (and the next test shows that the
    terms are needed)."""
    rng = np.random.default_rng(100 + L + int(spread))
    N = NT
    trials = 60 if L == 64 else 120
    accepted = 0
    for x, C, mu in _rows(rng, L, N, spread, trials, family):
        ok, ii, best = certify(x, C, mu, N, worst=True, GRP=GRP)
        if ok:
            accepted += 1
            assert ii == best, (ii, best)
    assert accepted > 0


@pytest.mark.parametrize("GRP,weights", [(2, w) for w in ({"m_R": 0}, {"m_R": 0.5}, {"m_k": 0},
                                                          {"m_k": 0.5}, {"m_pack": 0}, {"m_pack": 0.5},
                                                          {"m_E": 0}, {"m_E": 0.5}, {"lb_R": 0},
                                                          {"lb_E": 0}, {"lb_E": 0.5}, {"lb_pack": 0})] +
                                         [(8, w) for w in ({"m_R": 0}, {"m_k": 0}, {"m_E": 0},
                                                          {"lb_R": 0}, {"lb_E": 0}, {"lb_pack": 0})])
def test_bf16_certificate_terms_are_needed(GRP, weights):
    """With every error at its worst (as above), dropping or halving one term of
    the first certificate's margin, or dropping one of the second's lower bound,
    lets a wrong row through in one of the row families.  (Not shown this way:
    the eta terms, never binding here since x~ is exact for integer mu; halving
    R' in the second certificate, whose packing term leaves that much slack;
    with groups of eight, the first certificate's packing term, 2^-19 (|V1| +
    |V2|), for which the group's largest k' -- it stands in for the unknown k'
    of V1's member -- leaves more room than that in these families.)"""
    params = [(16, 20.0, "near"), (16, 2.0, "near"), (64, 20.0, "near"), (64, 2.0, "near"),
              (16, 0.5, "mirror"), (64, 0.5, "mirror")]
    for L, spread, family in params:
        rng = np.random.default_rng(100 + L + int(spread))
        trials = 60 if L == 64 else 120
        for x, C, mu in _rows(rng, L, NT, spread, trials, family):
            ok, ii, best = certify(x, C, mu, NT, worst=True, weights=weights, GRP=GRP)
            if ok and ii != best:
                return
    pytest.fail(f"weights {weights}: no wrong row accepted")


def test_bf16_certificates_accept_clear_winners():
    """With the accumulation error at the model's worst, a row next to one
    codevector of a spread codebook is still accepted."""
    rng = np.random.default_rng(5)
    L, N = 16, NT
    base = rng.integers(0, 256, L).astype(np.float32)
    C = (base + 40 * rng.standard_normal((N, L))).astype(np.float32)
    mu = np.rint(C.mean(0)).astype(np.float32)
    for n in rng.choice(N, 20, replace=False):
        x = np.clip(np.rint(C[n] + rng.standard_normal(L)), 0, 255).astype(np.float32)
        for GRP in (2, 4, 8):
            ok, ii, best = certify(x, C, mu, N, GRP=GRP)
            assert ok and ii == best == n


@pytest.mark.parametrize("GRP", [2, 4, 8])
def test_bf16_certificates_resolve_split_twins(GRP):
    """Right after a split every codevector has a twin at 2 delta (children 2i and 2i + 1 of
    the same parent).  Twins share a group, so the second-best value the certificates use
    comes from the next parent, and the twins themselves are told apart by their exact
    distances: rows near one parent are certified, each with its exact nearest twin."""
    rng = np.random.default_rng(17)
    L, N = 16, NT
    parents = (128 + 40 * rng.standard_normal((N // 2, L))).astype(np.float32)
    delta = np.float32(0.01)
    C = np.empty((N, L), np.float32)
    C[0::2] = parents + delta
    C[1::2] = parents - delta
    mu = np.rint(C.mean(0)).astype(np.float32)
    accepted = 0
    for n in rng.choice(N // 2, 24, replace=False):
        x = np.clip(np.rint(parents[n] + 3 * rng.standard_normal(L)), 0, 255).astype(np.float32)
        ok, ii, best = certify(x, C, mu, N, GRP=GRP)
        if ok:
            accepted += 1
            assert ii == best and best // 2 == n
    assert accepted >= 20


def _rows_real(rng, L, N, spread, trials):
    """Real-valued rows (not exact in BF16 after centring: the split form) with a
    near-tie pair as in _rows, codevectors around the row, an integer mu (the
    kernel rounds the centring vector)."""
    for trial in range(trials):
        x = (rng.random(L) + 0.3 * rng.standard_normal(L)).astype(np.float32)
        c0 = (x + spread * rng.standard_normal(L)).astype(np.float32)
        w = rng.standard_normal(L)
        w /= np.linalg.norm(w)
        d = c0.astype(np.float64) - x
        c1 = x + d - 2 * np.dot(d, w) * w
        eps = 0.0 if trial % 4 == 0 else spread * 10 ** rng.uniform(-7, 0)
        dv = rng.standard_normal(L)
        c1 = (c1 + eps * dv / np.linalg.norm(dv)).astype(np.float32)
        C = (x + spread * (2.5 + rng.standard_normal((N, L)))).astype(np.float32)
        p0 = 2 * int(rng.integers(0, N // 2))
        p1 = {0: p0 + 1, 1: (p0 + 6) % N, 2: (p0 + HALF + 3) % N}[trial % 3]
        C[p0], C[p1] = (c0, c1) if trial % 2 else (c1, c0)
        mu = np.rint(C.mean(0)).astype(np.float32)
        yield x, C, mu


@pytest.mark.parametrize("GRP", [2, 4, 8])
@pytest.mark.parametrize("L,spread", [(16, 0.2), (16, 0.02), (32, 0.2), (32, 0.02)])
def test_bf16_split_form_sound(L, spread, GRP):
    """Real-valued rows take the split form (x~ in two BF16 pieces, the remainder
    and the pieces' missed products bounded in E, X2 from the pieces): at the
    model's bound and with every bounded quantity at its worst, every accepted
    row has the exact argmin, and rows are accepted."""
    for worst in (False, True):
        rng = np.random.default_rng(300 + L + int(100 * spread) + (7 if worst else 0))
        accepted = 0
        for x, C, mu in _rows_real(rng, L, NT, spread, 60):
            assert not np.all((x - mu) == np.rint(x - mu))
            ok, ii, best = certify(x, C, mu, NT, worst=worst, GRP=GRP)
            if ok:
                accepted += 1
                assert ii == best, (ii, best)
        assert accepted > 0


def test_bf16_split_form_accepts_clear_winners():
    """Gaussian-mixture-like real data: a row near one codevector of a spread
    codebook is accepted in the split form."""
    rng = np.random.default_rng(21)
    L, N = 32, NT
    C = rng.random((N, L)).astype(np.float32)
    mu = np.rint(C.mean(0)).astype(np.float32)
    for n in rng.choice(N, 12, replace=False):
        x = (C[n] + 0.1 * rng.standard_normal(L)).astype(np.float32)
        for GRP in (2, 4, 8):
            ok, ii, best = certify(x, C, mu, N, GRP=GRP)
            assert ok and ii == best == n
