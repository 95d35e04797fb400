"""Pins of the oracle's BF16 reading of the learned proposal's network (the
reading of the library's tensor-core evaluators: BF16 inputs, weights, biases
and hidden activations, rounded to nearest with ties to even; sums exact).

Each check compares the oracle with something other than itself:
  * a network whose output has a closed form in the rounded values, with the
    BF16 rounding taken from numpy's round-half-even on the significand
    (frexp / rint / ldexp) rather than from the oracle's bit manipulation,
    and hand-derived values at rounding ties;
  * the slack of a rounding (distance to the nearest rounding boundary) on
    hand values and against the same numpy construction;
  * one learned move recomputed from the pinned pieces (features, draws,
    network) in the order the move takes them: the trial position and the
    acceptance margin must use the BF16 network both for the forward and the
    reverse density;
  * detailed balance of the move with the BF16 network by brute force on a
    dimer (exact for any proposal network, so it pins the wiring).
"""
import math

import numpy as np
import pytest

from paper_1711_03828_gb300 import SystemDesc, workloads
from tests.conftest import oracle_system
from tests.test_oracle_pins import check_two_particle_balance_brute_force


def bf16_ref(v):
    """Round-to-nearest-even of the FP32 value of v to 8 significant bits."""
    v = float(np.float32(v))
    if v == 0.0:
        return 0.0
    m, e = math.frexp(v)                  # v = m 2^e, 1/2 <= |m| < 1
    return math.ldexp(float(np.rint(m * 256.0)), e - 8)


def slack_ref(v, T):
    """Distance of the FP32 value v from the nearest BF16 rounding boundary, / T."""
    v = float(np.float32(v))
    if v == 0.0 or T <= 0.0:
        return math.inf
    m, e = math.frexp(abs(v))
    if math.ldexp(1.0, e - 8) < math.ldexp(T, -16):
        return math.inf
    q = m * 256.0                          # in [128, 256)
    bounds = [math.ldexp(math.floor(q - 0.5) + 0.5, e - 8),
              math.ldexp(math.floor(q - 0.5) + 1.5, e - 8),
              math.ldexp(127.75, e - 8)]   # between the binade below and this one
    return min(abs(abs(v) - b) for b in bounds) / T


# --------------------------------------------------------------------------
# A network with a closed form in the rounded values.  Layer 1 routes x_j and
# -x_j to separate units (weights 1 + 2^-9, which BF16 rounds to 1) and adds
# 3 * 2^-10; layer 2 is the identity (weights 1 + 2^-9) plus 5 * 2^-11; layer
# 3 sums with BF16-exact coefficients; output biases 0.1 k (rounded).  Every
# rounding site changes the output, so dropping any one of them is seen.
# --------------------------------------------------------------------------
def _hand_network():
    import oracle
    rng = np.random.default_rng(3)
    C = rng.integers(-8, 9, (4, 24)) / 8.0
    W = np.zeros(oracle.MLP_PARAMS)
    W1 = W[0:384].reshape(32, 12)
    b1 = W[384:416]
    W2 = W[416:1440].reshape(32, 32)
    b2 = W[1440:1472]
    W3 = W[1472:1600].reshape(4, 32)
    b3 = W[1600:1604]
    for j in range(12):
        W1[j, j] = 1.0 + 2.0**-9
        W1[12 + j, j] = -(1.0 + 2.0**-9)
    b1[:24] = 3.0 * 2.0**-10
    for j in range(24):
        W2[j, j] = 1.0 + 2.0**-9
    b2[:24] = 5.0 * 2.0**-11
    W3[:, :24] = C
    b3[:] = 0.1 * np.arange(4)
    return W, C


def _hand_network_want(C, x):
    xb = np.array([bf16_ref(v) for v in x])
    h1 = np.array([bf16_ref(max(z, 0.0)) for z in np.concatenate([xb, -xb]) + 3.0 * 2.0**-10])
    h2 = np.array([bf16_ref(max(z, 0.0)) for z in h1 + 5.0 * 2.0**-11])
    return C @ h2 + np.array([bf16_ref(0.1 * k) for k in range(4)])


def check_bf16_network_closed_form(lib=None):
    import oracle
    W, C = _hand_network()
    # hand values: 1 + 2^-8 and 1 + 3*2^-8 are ties (to 1 and 1 + 2^-6),
    # 1 + 3*2^-9 rounds up to 1 + 2^-7, 2^-20 stays exact
    assert bf16_ref(1 + 2.0**-8) == 1.0 and bf16_ref(1 + 3 * 2.0**-8) == 1 + 2.0**-6
    assert bf16_ref(1 + 3 * 2.0**-9) == 1 + 2.0**-7 and bf16_ref(-(1 + 2.0**-8)) == -1.0
    hand = [1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 3 * 2.0**-9, -(1 + 2.0**-8), 2.0**-20, 0.0,
            -3.14159, 2.71828, 0.1, -0.3, 7.77, -1e-3]
    rng = np.random.default_rng(5)
    for x in [np.array(hand)] + [rng.normal(size=12) * 3.0 for _ in range(20)]:
        got, _ = oracle.mlp_forward_bf16(W, x, L=lib)
        want = _hand_network_want(C, x)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
        # the FP64 reading of the same network differs (the roundings matter)
        assert np.max(np.abs(oracle.mlp_forward(W, x, L=lib) - want)) > 1e-5


def test_bf16_network_closed_form(oracle_lib):
    check_bf16_network_closed_form()


def check_bf16_slack_values(lib=None):
    import oracle
    s = lambda v, T: oracle.bf16_slack(v, T, L=lib)  # noqa: E731
    assert s(1 + 2.0**-8, 1.0) == 0.0                 # a rounding tie
    assert s(1.0, 1.0) == 2.0**-9                      # the boundary below 1 is 1 - 2^-9
    assert s(1.5, 1.0) == 2.0**-8                      # spacing 2^-7 in [1, 2)
    assert s(-1.5, 2.0) == 2.0**-9                     # sign-symmetric, in units of T
    assert s(0.0, 1.0) == math.inf and s(1.0, 0.0) == math.inf
    assert s(1.0, 2.0**10) == math.inf                 # spacing 2^-7 < 2^-16 T: negligible
    rng = np.random.default_rng(9)
    v = (rng.normal(size=3000) * np.exp(rng.uniform(-8, 8, 3000))).astype(np.float32)
    T = np.abs(v.astype(np.float64)) * np.exp(rng.uniform(-2, 2, 3000))
    for a, t in zip(v, T):
        want = slack_ref(float(a), float(t))
        assert s(float(a), float(t)) == pytest.approx(want, rel=1e-12, abs=0.0), (a, t)
    # a value moved by its slack (in units of T) reaches a boundary: it rounds
    # differently a few FP32 ulps past it
    for a, t in zip(v[:300], T[:300]):
        sl = s(float(a), float(t))
        if not math.isfinite(sl):
            continue
        a64 = float(a)
        step = sl * t + 4.0 * float(np.spacing(np.float32(abs(a))))
        up, dn = a64 + step, a64 - step
        assert bf16_ref(up) != bf16_ref(a64) or bf16_ref(dn) != bf16_ref(a64)


def test_bf16_slack_values(oracle_lib):
    check_bf16_slack_values()


# --------------------------------------------------------------------------
# One learned move rebuilt from the pinned pieces (fixed even -> odd order, so
# every even particle moves first with both partners at their old positions).
# --------------------------------------------------------------------------
def check_bf16_move_uses_the_bf16_network(lib=None):
    import oracle
    from oracle import Positions
    d = SystemDesc(n_chains=24, N=8, f=0.5, box_Re=(1.0, 1.0, 1.0), grid=(6, 6, 6), chiN=25.0,
                   kappaN=50.0, move=2, set_order=1, seed=29)
    s = oracle_system(d, lib)
    W = workloads.random_mlp(15, scale=0.3)
    W[:384] *= 1.0 + 2.0**-10           # weights that BF16 must round
    s.set_mlp(W, bf16=True)
    pos0 = workloads.random_walk_positions(d, seed=31)
    p = Positions(pos0[0].copy(), pos0[1].copy(), pos0[2].copy())
    before = p.copy()
    nA, nB = s.histogram(p)
    wA, wB = s.fields(nA, nB)
    sweep = 7
    _, margin, acc, trial, slack = s.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True,
                                           want_trial=True, want_slack=True)
    P = s.params
    sigma0 = P.a / math.sqrt(3.0)
    n_diff = 0
    for chain in range(d.n_chains):
        for i in range(0, d.N, 2):
            m = chain * d.N + i
            w_t = wA if i < P.N_A else wB
            r = np.array([before.x[m], before.y[m], before.z[m]], np.float64)
            w1 = s.draw(1, m, sweep)
            w2 = s.draw(2, m, sweep)
            u = [((int(v) >> 8) + 0.5) / 2**24 for v in w1]
            xi = []
            for k in range(2):
                rad, th = math.sqrt(-2.0 * math.log(u[2 * k])), 2.0 * math.pi * u[2 * k + 1]
                xi += [rad * math.cos(th), rad * math.sin(th)]
            f = s.learned_features(before, w_t, chain, i, r)
            o, _ = oracle.mlp_forward_bf16(W, f, L=lib)
            sig = sigma0 * math.exp(2.0 * math.tanh(0.5 * o[3]))
            rp = np.array([float(np.float32(r[k] + float(np.float32(o[k] + sig * xi[k]))))
                           for k in range(3)])
            assert np.array_equal(trial[:, m].astype(np.float64), rp), (m, trial[:, m], rp)
            fr = s.learned_features(before, w_t, chain, i, rp)
            orv, _ = oracle.mlp_forward_bf16(W, fr, L=lib)
            sigr = sigma0 * math.exp(2.0 * math.tanh(0.5 * orv[3]))
            nb = [n for n in (m - 1, m + 1) if 0 <= n - chain * d.N < d.N]
            Kb = P.K_b
            dE = sum(Kb * (np.sum((rp - [before.x[n], before.y[n], before.z[n]]) ** 2)
                           - np.sum((r - [before.x[n], before.y[n], before.z[n]]) ** 2)) for n in nb)
            cell = lambda q: int(((math.floor(q[2]) % 6) * 6 + math.floor(q[1]) % 6) * 6  # noqa: E731
                                 + math.floor(q[0]) % 6)
            dE += w_t[cell(rp)] - w_t[cell(r)]
            lq_f = -np.sum((rp - r - o[:3]) ** 2) / (2 * sig * sig) - 3 * math.log(sig)
            lq_r = -np.sum((r - rp - orv[:3]) ** 2) / (2 * sigr * sigr) - 3 * math.log(sigr)
            la = -dE + lq_r - lq_f
            lnu = math.log(((int(w2[0]) >> 8) + 0.5) / 2**24)
            assert margin[m] == pytest.approx(lnu - la, rel=1e-9, abs=1e-9), m
            assert acc[m] == int(la >= 0.0 or lnu < la)
            assert 0.0 <= slack[m] < math.inf
            # the FP64 network proposes elsewhere
            of = oracle.mlp_forward(W, f, L=lib)
            n_diff += int(np.max(np.abs(of - o)) > 1e-6)
    assert n_diff > 0.9 * d.n_chains * d.N / 2


def test_bf16_move_uses_the_bf16_network(oracle_lib):
    check_bf16_move_uses_the_bf16_network()


@pytest.mark.parametrize("set_order", [0, 1])
def test_bf16_learned_move_balance_brute_force(oracle_lib, set_order):
    check_two_particle_balance_brute_force(set_order, move=2, bf16=True)
