"""The error bound behind the fast policy's FP32 screen of the restriction test (Eq. (be_res))
and of theta (Eq. (tau_we6)).

The fast arithmetic policy first forms the four indicators and tau5, tau6 of a stencil in
FP32, from the high 32 bits of the FP64 differences, and takes the decisions there only when
an error bound proves that the FP64 evaluation decides the same.  This test restates that
screen with numpy (the same truncation, FP32 operations and margins) and checks the claim
itself: on smooth, random, step, polynomial, constant and near-threshold stencils, and on
stencils within 1e-12 .. 1e-5 of either decision boundary (one family with an indicator that
vanishes by cancellation, where the absolute error bound matters), for the
alpha_R values the paper uses, every decision the screen takes agrees with the FP64
decision; and inputs out of its range, or not finite, are left to FP64.  It runs on the CPU.
"""
import numpy as np
import pytest

F32 = np.float32


def hi32(x):
    """Sign, rebiased exponent and the top 20 mantissa bits of each double, as a float32;
    0 below 2^-126."""
    hi = (np.asarray(x, dtype=np.float64).view(np.uint64) >> np.uint64(32)).astype(np.int64)
    mag = hi & 0x7FFFFFFF
    fb = (((mag - 0x38000000) << 3) & 0xFFFFFFFF) | (hi & 0x80000000)
    out = fb.astype(np.uint32).view(np.float32).copy()
    out[mag < 0x38100000] = 0.0
    return out


def high_word(x):
    return (np.asarray(x, dtype=np.float64).view(np.uint64) >> np.uint64(32)).astype(np.int64) & 0x7FFFFFFF


def fmaf(a, b, c):
    # a*b is exact in float64 for float32 operands; one rounding to float32 after the add
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def differences(q):
    d = np.diff(q, axis=1)
    s = np.diff(d, axis=1)
    d0, d1, d2, d3, d4 = d.T
    s0, s1, s2, s3 = s.T
    t5b = s2 - s1
    t5a = (-2.0 * s1 + s0) + s2
    t6a = -3.0 * t5b + (s3 - s0)
    t6b = (s0 + s3) - (s1 + s2)
    return (s0, s1, s2, s3, d1, d2, d3, t5a, t5b, t6a, t6b)


def decide_fp64(args, eps, alpha_r):
    """The restriction and theta decisions in binary64 (Eqs. (be0_cen)-(be3_cen), (be_res),
    (tau_5), (tau_6), (tau_we6))."""
    s0, s1, s2, s3, d1, d2, d3, t5a, t5b, t6a, t6b = args
    e0, g3, e3 = s0 + d1, 3.0 * s2 - s3, s3 - d3
    b = np.stack([13 / 12 * s0 * s0 + e0 * e0, 13 / 12 * s1 * s1 + d2 * d2, 13 / 12 * s2 * s2 + d2 * d2,
                  13 / 48 * g3 * g3 + e3 * e3])
    restricted = b.max(axis=0) <= alpha_r * (eps + b.min(axis=0))
    tau5 = 13 / 12 * t5a * t5a + t5b * t5b
    tau6 = 13 / 12 * t6a * t6a + 0.25 * (t6b * t6b)
    theta1 = ~(tau6 < tau5)
    return restricted, theta1


def screen(args, eps, alpha_r):
    """0: left to FP64; 1: restricted with theta = 1; 2: restricted with theta = 0."""
    s0, s1, s2, s3, d1, d2, d3, t5a, t5b, t6a, t6b = args
    hm = np.max(np.stack([high_word(v) for v in args] + [np.full(s0.shape, high_word(np.array([alpha_r]))[0])]),
                axis=0)
    in_range = hm < 0x43B00000  # every input below 2^60 and finite
    a0, a1, a2, a3 = (hi32(v) for v in (s0, s1, s2, s3))
    x1, x2, x3 = (hi32(v) for v in (d1, d2, d3))
    f1312, f1348 = F32(13 / 12), F32(13 / 48)
    e0, g3, e3, dd = a0 + x1, fmaf(F32(3), a2, -a3), a3 - x3, x2 * x2
    b = np.stack([fmaf(f1312 * a0, a0, e0 * e0), fmaf(f1312 * a1, a1, dd), fmaf(f1312 * a2, a2, dd),
                  fmaf(f1348 * g3, g3, e3 * e3)])
    sg = np.max(np.abs(np.stack([a0, a1, a2, a3, x1, x2, x3])), axis=0)
    dl = F32(2.0 ** -14) * (sg * sg)
    ar, ef = hi32(np.array([alpha_r]))[0], hi32(np.array([eps]))[0]
    scale_ok = ar * ef > F32(1e-30)
    sure = (b.max(axis=0) + dl) < ar * (ef + (b.min(axis=0) - dl)) * F32(1 - 2.0 ** -18)
    u5a, u5b, u6a, u6b = (hi32(v) for v in (t5a, t5b, t6a, t6b))
    tau5 = fmaf(f1312 * u5a, u5a, u5b * u5b)
    tau6 = fmaf(f1312 * u6a, u6a, F32(0.25) * (u6b * u6b))
    tm = np.maximum(tau5, tau6)
    theta_sure = (tm > F32(2.0 ** -120)) & (np.abs(tau6 - tau5) > F32(2.0 ** -16) * tm)
    all_zero = np.all(np.stack([(np.asarray(v).view(np.uint64) << np.uint64(1)) == 0 for v in (t5a, t5b, t6a, t6b)]),
                      axis=0)
    out = np.zeros(s0.shape, dtype=np.int64)
    go = in_range & scale_ok & sure
    out[go & theta_sure] = np.where(tau6 < tau5, 2, 1)[go & theta_sure]
    out[go & ~theta_sure & all_zero] = 1
    return out


def stencils(rng, n):
    x = np.arange(6.0)[None, :]
    out = []
    for dx in (1e-1, 1e-2, 2.4e-3, 1e-4):  # smooth data, amplitudes 1e-6 .. 1e2
        x0, k, amp = rng.uniform(-5, 5, (n, 1)), rng.uniform(1, 8, (n, 1)), 10 ** rng.uniform(-6, 2, (n, 1))
        out.append(("smooth", amp * np.sin(k * (x0 + dx * x)) + rng.uniform(-1, 1, (n, 1))))
    out.append(("random", rng.normal(size=(n, 6)) * 10 ** rng.uniform(-8, 3, (n, 1))))
    out.append(("step", np.where(x < rng.integers(0, 7, (n, 1)), rng.uniform(0, 1, (n, 1)), rng.uniform(0, 1, (n, 1)))))
    out.append(("linear", rng.uniform(-1, 1, (n, 1)) + rng.uniform(-1, 1, (n, 1)) * x))
    out.append(("quadratic", rng.uniform(-1, 1, (n, 1)) + rng.uniform(-1, 1, (n, 1)) * x
                + rng.uniform(-1, 1, (n, 1)) * x ** 2 * 10 ** rng.uniform(-6, 0, (n, 1))))
    out.append(("constant", np.repeat(rng.uniform(-1, 1, (n, 1)), 6, axis=1)))
    out.append(("noise on a constant", rng.uniform(-1, 1, (n, 1)) + 1e-14 * rng.normal(size=(n, 6))))
    near = rng.normal(size=(n, 6))
    near[:, 3:] *= rng.uniform(0.5, 5, (n, 1))
    out.append(("near the restriction threshold", near))
    return out


def boundary_stencils(rng, n, eps, alpha_r, which):
    """Stencils q = u + lam v within a relative 1e-12 .. 1e-5 of a point where the FP64
    restriction test (which = 0, 2) or the sign of tau6 - tau5 (which = 1) changes."""

    def f(lam, u, v):
        args = differences(u + lam[:, None] * v)
        if which == 0:
            s0, s1, s2, s3, d1, d2, d3 = args[:7]
            e0, g3, e3 = s0 + d1, 3.0 * s2 - s3, s3 - d3
            b = np.stack([13 / 12 * s0 * s0 + e0 * e0, 13 / 12 * s1 * s1 + d2 * d2, 13 / 12 * s2 * s2 + d2 * d2,
                          13 / 48 * g3 * g3 + e3 * e3])
            return b.max(axis=0) - alpha_r * (eps + b.min(axis=0))
        t5a, t5b, t6a, t6b = args[7:]
        return (13 / 12 * t6a * t6a + 0.25 * (t6b * t6b)) - (13 / 12 * t5a * t5a + t5b * t5b)

    u = rng.normal(size=(n, 6)) * 10 ** rng.uniform(-3, 2, (n, 1))
    if which == 2:
        # beta_3 = 0 through cancellation (3 s2 = s3 = d3: differences a, 1.5a, 3a on the
        # right), the other indicators of the size of the largest input: near the boundary
        # beta_3 is small against that size, where the absolute error bound matters
        a = rng.uniform(0.5, 2.0, (n, 1)) * rng.choice([-1.0, 1.0], (n, 1))
        d = np.concatenate([rng.normal(size=(n, 2)), a, 1.5 * a, 3.0 * a], axis=1)
        u = np.concatenate([np.zeros((n, 1)), np.cumsum(d, axis=1)], axis=1) * 10 ** rng.uniform(-2, 2, (n, 1))
        which = 0
    v = rng.normal(size=(n, 6)) * 10 ** rng.uniform(-3, 2, (n, 1)) * (np.abs(u).max(axis=1, keepdims=True) + 1e-3)
    lo, hi = np.zeros(n), np.ones(n)
    flo, fhi = f(lo, u, v), f(hi, u, v)
    keep = np.sign(flo) != np.sign(fhi)
    u, v, lo, hi, flo = u[keep], v[keep], lo[keep], hi[keep], flo[keep]
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        fm = f(mid, u, v)
        same = np.sign(fm) == np.sign(flo)
        lo, hi = np.where(same, mid, lo), np.where(same, hi, mid)
        flo = np.where(same, fm, flo)
    lam = 0.5 * (lo + hi)
    k = len(lam)
    off = rng.choice([-1.0, 1.0], k) * 10 ** rng.uniform(-12, -5, k) * np.maximum(lam, 1e-3)
    return u + (lam + off)[:, None] * v


@pytest.mark.parametrize("alpha_r", [1.0, 10.0, 50.0])
def test_screened_decisions_equal_the_fp64_decisions(alpha_r):
    rng = np.random.default_rng(int(alpha_r))
    eps = 1e-10
    decided_smooth = []
    for label, q in stencils(rng, 40000):
        args = differences(q)
        restricted, theta1 = decide_fp64(args, eps, alpha_r)
        with np.errstate(all="ignore"):
            sc = screen(args, eps, alpha_r)
        taken = sc > 0
        wrong = taken & (~restricted | ((sc == 1) != theta1))
        assert not wrong.any(), (label, alpha_r, int(wrong.sum()))
        if label == "smooth":
            decided_smooth.append(taken[restricted].mean())
    for which in (0, 1, 2):  # at the two decision boundaries, where the margins matter
        q = boundary_stencils(rng, 40000, eps, alpha_r, which)
        args = differences(q)
        restricted, theta1 = decide_fp64(args, eps, alpha_r)
        with np.errstate(all="ignore"):
            sc = screen(args, eps, alpha_r)
        taken = sc > 0
        wrong = taken & (~restricted | ((sc == 1) != theta1))
        assert not wrong.any(), ("boundary", which, alpha_r, int(wrong.sum()))
    if alpha_r >= 10.0:
        # the bound is not so loose as to be useless: restricted smooth stencils are decided
        assert min(decided_smooth) > 0.99, decided_smooth


def test_out_of_range_and_non_finite_inputs_are_left_to_fp64():
    eps, alpha_r = 1e-10, 10.0
    q = np.array([[0.0, 1.0, 2.0, 3.0, 4.0, 5.0]] * 4)
    q[0] *= 2.0 ** 61  # differences beyond 2^60
    q[1, 2] = np.inf
    q[2, 3] = np.nan
    q[3] = 1.0  # constant: decided, restricted with theta = 1 (a tie of tau5 = tau6 = 0)
    with np.errstate(all="ignore"):
        sc = screen(differences(q), eps, alpha_r)
    assert sc[:3].tolist() == [0, 0, 0]
    assert sc[3] == 1
    # alpha_R * eps below the screen's range: everything is left to FP64
    sc = screen(differences(np.cumsum(np.ones((3, 6)), axis=1) ** 2), 1e-40, alpha_r)
    assert (sc == 0).all()


def test_hi32_truncates_within_two_to_the_minus_twenty():
    rng = np.random.default_rng(5)
    x = rng.normal(size=100000) * 10 ** rng.uniform(-30, 17, 100000)
    f = hi32(x).astype(np.float64)
    assert np.all(np.abs(f - x) <= 2.0 ** -20 * np.abs(x))
    assert np.all(np.sign(f) == np.sign(x))
    assert hi32(np.array([1e-39]))[0] == 0.0 and hi32(np.array([0.0]))[0] == 0.0
