"""Learned MH-corrected proposal: training gradient and sweep against the FP64
oracle, exactness by brute force on the GPU, and the gain of training.

Training gradient (FP32 weights): per-sample J and log alpha to 1e-5 relative
(1e-5 absolute), the gradient summed over samples to 1e-4 of its norm;
samples whose trial position lies within 1e-4 dL of a cell face or whose log
alpha is within 1e-3 of the kink of min(1, e^l) are left out (there the FP32
and FP64 evaluations may take different branches).
Sweep: one cycle from the same positions and BF16-exact random weights, the
tolerances of the smart Monte Carlo move (the network and the normals are
evaluated in FP32 on the GPU, in FP64 in the oracle), with the FP32 network
(SOMA_FLAG_LEARNED_FP32).  The tensor-core networks (the default mma.sync one
and the tcgen05 one; BF16 operands and activations, FP32 sums) against the
oracle's BF16 reading of the network, one cycle element by element; they are
also checked for exactness by brute force and against each other.
"""
import math

import numpy as np
import pytest

from oracle import Positions
from paper_1711_03828_gb300 import (FLAG_LEARNED_FP32, FLAG_LEARNED_UMMA, MOVE_LEARNED,
                                    MOVE_SMC, System, SystemDesc, workloads)
from tests.conftest import oracle_system
from tests.test_gpu_parity import _pos
from tests.test_gpu_smc import _near_face, _tol

pytestmark = pytest.mark.gpu

TIE_LEARNED = 1e-3


def _state(d, seed):
    pos0 = workloads.random_walk_positions(d, seed=seed)
    s = System(d)
    s.set_positions(pos0)
    s.update_fields()
    orc = oracle_system(d)
    p = _pos(pos0)
    nA, nB = orc.histogram(p)
    wA, wB = orc.fields(nA, nB)
    return s, orc, p, wA, wB


def test_training_gradient_matches_oracle(cuda_device):
    d = workloads.melt_small(n_chains=256, chiN=30.0, move=MOVE_LEARNED)
    s, orc, p, wA, wB = _state(d, 21)
    W = workloads.random_mlp(11).astype(np.float32)
    rng = np.random.default_rng(4)
    n = 512
    samples = np.stack([rng.integers(0, d.n_chains, n), rng.integers(0, d.N, n)], 1).astype(np.uint32)
    xi = rng.normal(size=(n, 3)).astype(np.float32)
    _, J, la = s.proposal_grad(samples, xi, w=W)
    Wd = W.astype(np.float64)
    keep = []
    for b in range(n):
        Jo, _, lo = orc.esjd_sample(Wd, p, wA, wB, samples[b, 0], samples[b, 1], xi[b].astype(np.float64),
                                    want_grad=False)
        # trial position of the oracle (no FP32 rounding), for the face check
        f = orc.learned_features(p, wA if samples[b, 1] < orc.params.N_A else wB, samples[b, 0],
                                 samples[b, 1],
                                 [p.x[samples[b, 0] * d.N + samples[b, 1]],
                                  p.y[samples[b, 0] * d.N + samples[b, 1]],
                                  p.z[samples[b, 0] * d.N + samples[b, 1]]])
        import oracle as O
        o = O.mlp_forward(Wd, f)
        sig = orc.params.a / math.sqrt(3) * math.exp(2 * math.tanh(0.5 * o[3]))
        m = samples[b, 0] * d.N + samples[b, 1]
        rp = np.array([p.x[m], p.y[m], p.z[m]], np.float64) + o[:3] + sig * xi[b]
        near = np.any(np.abs(rp - np.round(rp)) < 1e-4)
        if near or abs(lo) < 1e-3:
            continue
        assert abs(J[b] - Jo) <= 1e-5 * max(1.0, abs(Jo)), (b, J[b], Jo)
        assert abs(la[b] - lo) <= 1e-4 * max(1.0, abs(lo)), (b, la[b], lo)
        keep.append(b)
    assert len(keep) > 0.8 * n
    keep = np.asarray(keep)
    g_gpu, _, _ = s.proposal_grad(samples[keep], xi[keep], w=W)
    g_or = np.zeros(1604)
    for b in keep:
        _, g, _ = orc.esjd_sample(Wd, p, wA, wB, samples[b, 0], samples[b, 1],
                                  xi[b].astype(np.float64))
        g_or += g
    err = np.linalg.norm(g_gpu - g_or) / np.linalg.norm(g_or)
    print(f"training gradient over {len(keep)} samples: relative error {err:.2e}")
    assert err < 1e-4
    s.close()


@pytest.mark.parametrize("N,n_chains,grid,box", [
    (32, 1024, (12, 12, 12), (2.0, 2.0, 2.0)),
    (7, 1500, (9, 9, 6), (1.5, 1.5, 1.0)),
    (64, 512, (12, 12, 12), (2.0, 2.0, 2.0)),
])
def test_learned_one_cycle_matches_oracle(cuda_device, N, n_chains, grid, box):
    d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=box, grid=grid, chiN=30.0,
                   kappaN=50.0, move=MOVE_LEARNED, seed=11, flags=FLAG_LEARNED_FP32)
    W = workloads.random_mlp(5, scale=0.2)
    moves = mism = accepted = 0
    for k, sweep in enumerate((0, 3, 1000)):
        pos0 = workloads.random_walk_positions(d, seed=300 + k)
        orc = oracle_system(d)
        orc.set_mlp(W)
        s = System(d)
        s.set_proposal_weights(W.astype(np.float32))
        s.set_positions(pos0)
        s.set_sweep(sweep)
        p = _pos(pos0)
        nA, nB = orc.histogram(p)
        wA, wB = orc.fields(nA, nB)
        _, margin, acc, trial = orc.sweep(p, wA, wB, sweep, want_margin=True, want_acc=True,
                                          want_trial=True)
        s.sweep(1)
        g = s.get_positions()
        s.close()
        gacc = np.any(g != pos0, axis=0).astype(np.uint8)
        bad = np.nonzero(gacc != acc)[0]
        ok = set(bad[np.abs(margin[bad]) < TIE_LEARNED].tolist())
        face = _near_face(trial)
        ok |= {int(m) for m in bad if face[m]}
        for m in bad.tolist():
            if m not in ok:
                assert any(k2 in ok and k2 // d.N == m // d.N for k2 in (m - 1, m + 1)), (m, margin[m])
        keep = np.ones(d.n_chains, bool)
        keep[np.unique(bad // d.N)] = False
        keep = np.repeat(keep, d.N)
        np.testing.assert_array_equal(g[:, keep & (acc == 0)], pos0[:, keep & (acc == 0)])
        sel = keep & (acc == 1)
        err = np.abs(g[:, sel].astype(np.float64) - trial[:, sel]) / _tol(trial[:, sel])
        assert err.max(initial=0) <= 1.0, err.max()
        moves += d.M
        mism += len(bad)
        accepted += int(acc.sum())
    print(f"learned N={N}: {moves} moves, acceptance {accepted / moves:.3f}, mismatches {mism}")
    assert mism <= max(3, 5e-4 * moves)


# A BF16 rounding of the tensor-core network may round the other way on the
# GPU, whose sums are FP32 in the tensor cores' own order, when the oracle's
# exact value lies within this fraction of the magnitude of its terms from a
# rounding boundary: a sum of K <= 32 products and the accumulator whose
# alignment truncates errs by at most (K + 1) 2^-23 of the terms' magnitude,
# below 2^-17 (and the trial position, fed back as features, inherits it).
SLACK_BF16 = 2.0**-17


@pytest.mark.parametrize("flags", [0, FLAG_LEARNED_UMMA], ids=["mma_sync", "tcgen05"])
@pytest.mark.parametrize("N,n_chains,grid,box", [
    (32, 1001, (12, 12, 12), (2.0, 2.0, 2.0)),
    (64, 257, (12, 12, 9), (2.0, 2.0, 1.5)),
    (2, 4099, (6, 6, 6), (1.0, 1.0, 1.0)),
    (8, 1003, (12, 12, 12), (2.0, 2.0, 2.0)),
])
def test_learned_tensor_core_one_cycle_matches_bf16_oracle(cuda_device, N, n_chains, grid, box,
                                                           flags):
    """The default learned sweep (BF16 network on the tensor cores, mma.sync)
    and the tcgen05 one against the oracle's BF16 reading of the network, one
    cycle from the same state, element by element.  Weights that BF16 must
    round.  Tolerances of the smart Monte Carlo move, except that a move
    whose oracle evaluation has a rounding within SLACK_BF16 of a BF16
    boundary (or whose bonded partner's has) may round differently and so
    propose up to 1e-2 dL elsewhere; such deviations must stay rare.  Chain
    counts leave ragged last tiles and blocks with fewer than four tiles."""
    d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=box, grid=grid, chiN=30.0,
                   kappaN=50.0, move=MOVE_LEARNED, seed=11, flags=flags)
    W = workloads.random_mlp(5, scale=0.2) * (1.0 + 2.0**-10)
    moves = mism = accepted = flagged = deviating = 0
    for k, sweep in enumerate((0, 3, 1000)):
        pos0 = workloads.random_walk_positions(d, seed=300 + k)
        orc = oracle_system(d)
        orc.set_mlp(W, bf16=True)
        s = System(d)
        s.set_proposal_weights(W.astype(np.float32))
        s.set_positions(pos0)
        s.set_sweep(sweep)
        p = _pos(pos0)
        nA, nB = orc.histogram(p)
        wA, wB = orc.fields(nA, nB)
        _, margin, acc, trial, slack = orc.sweep(p, wA, wB, sweep, want_margin=True,
                                                 want_acc=True, want_trial=True, want_slack=True)
        s.sweep(1)
        g = s.get_positions()
        s.close()
        near = slack < SLACK_BF16
        same_chain = lambda a, b: a // N == b // N  # noqa: E731
        expl = near.copy()
        expl[1:] |= near[:-1] & same_chain(np.arange(1, d.M), np.arange(d.M - 1))
        expl[:-1] |= near[1:] & same_chain(np.arange(d.M - 1), np.arange(1, d.M))
        gacc = np.any(g != pos0, axis=0).astype(np.uint8)
        bad = np.nonzero(gacc != acc)[0]
        ok = set(bad[np.abs(margin[bad]) < TIE_LEARNED].tolist())
        face = _near_face(trial)
        ok |= {int(m) for m in bad if face[m] or expl[m]}
        for m in bad.tolist():
            if m not in ok:
                assert any(k2 in ok and k2 // N == m // N for k2 in (m - 1, m + 1)), \
                    (m, margin[m], slack[m])
        keep = np.ones(d.n_chains, bool)
        keep[np.unique(bad // N)] = False
        keep = np.repeat(keep, N)
        np.testing.assert_array_equal(g[:, keep & (acc == 0)], pos0[:, keep & (acc == 0)])
        sel = keep & (acc == 1)
        dev = np.max(np.abs(g.astype(np.float64) - trial), axis=0)
        # the normals (hardware log and sincos) err by ~2^-21 of the step, so
        # the SMC tolerance grows with the step where it exceeds 3 dL (N = 2:
        # steps up to ~13 dL)
        step = np.max(np.abs(trial - pos0.astype(np.float64)), axis=0)
        strict = dev <= np.maximum(_tol(trial[0]), 2e-6 * step)
        off = np.nonzero(sel & ~strict)[0]
        unexplained = off[~expl[off]]
        assert len(unexplained) == 0, (unexplained[:10], dev[unexplained[:10]], slack[unexplained[:10]])
        assert dev[off].max(initial=0) <= 1e-2, dev[off].max()
        moves += d.M
        mism += len(bad)
        accepted += int(acc.sum())
        flagged += int(near.sum())
        deviating += len(off)
    print(f"learned tensor-core network (flags={flags}) N={N}: {moves} moves, acceptance "
          f"{accepted / moves:.3f}, decision mismatches {mism}, moves near a BF16 boundary "
          f"{flagged}, proposals off by more than 1e-6 R_e0 {deviating}")
    assert accepted > 0.05 * moves
    assert mism <= max(3, 1e-3 * moves)
    assert deviating <= max(3, 1e-2 * moves)


@pytest.mark.parametrize("N,n_chains", [(32, 1000), (2, 4099), (64, 257)])
def test_tcgen05_network_matches_mma_sync_network(cuda_device, N, n_chains):
    """The tcgen05 evaluator (one M = 128 product per layer over a 4-warp
    block, accumulator in tensor memory) and the warp-level mma.sync evaluator
    take the same BF16 operands and accumulate in FP32; only the summation
    order inside the tensor cores differs.  One cycle from the same state and
    weights: every decision agrees except at near-ties, and every position
    agrees to 2e-6 dL (a few FP32 ulps of the network output).  Chain counts
    leave ragged last tiles and blocks with fewer than four tiles."""
    box = (2.0, 2.0, 1.5) if N > 2 else (1.0, 1.0, 1.0)
    grid = (12, 12, 9) if N > 2 else (6, 6, 6)
    W = workloads.random_mlp(9, scale=0.2).astype(np.float32)
    out = []
    for flags in (FLAG_LEARNED_UMMA, 0):
        d = SystemDesc(n_chains=n_chains, N=N, f=0.5, box_Re=box, grid=grid, chiN=30.0,
                       kappaN=50.0, move=MOVE_LEARNED, seed=13, flags=flags)
        pos0 = workloads.random_walk_positions(d, seed=77)
        s = System(d)
        s.set_proposal_weights(W)
        s.set_positions(pos0)
        s.update_fields()
        s.sweep(1)
        out.append((pos0, s.get_positions(), s.observables()["accepted"]))
        s.close()
    (p0, a, na), (_, b, nb) = out
    moved_a, moved_b = np.any(a != p0, axis=0), np.any(b != p0, axis=0)
    differ = np.nonzero(moved_a != moved_b)[0]
    close = np.all(np.abs(a.astype(np.float64) - b) <= 2e-6 * np.maximum(1.0, np.abs(a)), axis=0)
    print(f"N={N}: {a.shape[1]} moves, accepted {na} / {nb}, decisions differ {len(differ)}, "
          f"positions beyond 2e-6: {int((~close).sum())}")
    assert len(differ) <= max(2, 2e-4 * a.shape[1])
    # a different decision changes that particle and, through its new position,
    # at most the later move of its bonded partners
    assert (~close).sum() <= 3 * len(differ) + max(2, 2e-4 * a.shape[1])
    assert na > 0.05 * a.shape[1]


def _pair_probabilities(K, L):
    from tests.test_oracle_pins import _pair_cell_probabilities
    z = np.zeros(L**3)
    return _pair_cell_probabilities(K, L, z, z)


@pytest.mark.parametrize("move,flags", [(0, 0), (MOVE_SMC, 0), (MOVE_LEARNED, 0),
                                        (MOVE_LEARNED, FLAG_LEARNED_UMMA),
                                        (MOVE_LEARNED, FLAG_LEARNED_FP32)])
def test_gpu_two_particle_balance_brute_force(cuda_device, move, flags):
    """Dimers with chiN = kappaN = 0 on a periodic 2^3 grid: the visited cell
    pairs follow the exact distribution (erf quadrature) for every move type,
    the learned one with random weights (a strongly asymmetric proposal)."""
    L, Re = 2, 1.5
    d = SystemDesc(n_chains=16384, N=2, f=0.5, box_Re=(L / Re,) * 3, grid=(L,) * 3, chiN=0.0,
                   kappaN=0.0, move=move, seed=23, flags=flags)
    s = System(d)
    if move == MOVE_LEARNED:
        s.set_proposal_weights(workloads.random_mlp(7, scale=0.1).astype(np.float32))
    s.sweep(100)
    T = 400
    counts = np.zeros((d.n_chains, L**6))
    for _ in range(T):
        s.sweep(1)
        P = s.get_positions().reshape(3, d.n_chains, 2).astype(np.float64)
        c = np.floor(P).astype(np.int64) % L
        ci = (c[2] * L + c[1]) * L + c[0]
        counts[np.arange(d.n_chains), ci[:, 0] * L**3 + ci[:, 1]] += 1
    s.close()
    K = 3.0 / (2 * Re * Re)
    Pex = _pair_probabilities(K, L).reshape(-1)
    freq = counts / T
    est = freq.mean(0)
    se = freq.std(0) / math.sqrt(d.n_chains)
    z = (est - Pex) / np.maximum(se, 1e-12)
    print(f"move {move}: max |z| {np.max(np.abs(z)):.2f}")
    assert np.max(np.abs(z)) < 5.0


def test_training_increases_the_expected_jump(cuda_device):
    """Training on plain-method configurations raises the mean accepted squared
    displacement per move of the learned proposal above that of the untrained
    (zero-weight Gaussian) proposal, measured over whole sweeps."""
    d = workloads.melt_small(chiN=20.0, move=MOVE_LEARNED)

    def msd_per_move(s, sweeps=20):
        tot = 0.0
        for _ in range(sweeps):
            a = s.get_positions().astype(np.float64)
            s.sweep(1)
            b = s.get_positions().astype(np.float64)
            tot += ((b - a) ** 2).sum() / d.M
        return tot / sweeps

    base = System(d)
    base.sweep(50)
    msd0 = msd_per_move(base)
    base.close()
    s = System(d)
    log = s.train_proposal(steps=300, batch=8192, sweeps_between=1, lr=3e-3)
    msd1 = msd_per_move(s)
    s.close()
    uni = System(workloads.melt_small(chiN=20.0))
    uni.sweep(50)
    msd_u = msd_per_move(uni)
    uni.close()
    # the same trained weights through the FP32 network
    W = None
    f32 = System(workloads.melt_small(chiN=20.0, move=MOVE_LEARNED, flags=FLAG_LEARNED_FP32))
    s2 = System(d)
    s2.train_proposal(steps=300, batch=8192, sweeps_between=1, lr=3e-3)
    W = s2.get_proposal_weights()
    s2.close()
    f32.set_proposal_weights(W)
    f32.sweep(50)
    msd2 = msd_per_move(f32)
    f32.close()
    print(f"training: J {log['mean_J_first']:.4f} -> {log['mean_J_last']:.4f}, "
          f"alpha {log['mean_alpha_last']:.3f}; msd/move untrained {msd0:.4f}, "
          f"trained {msd1:.4f} (tensor cores) {msd2:.4f} (FP32 network), uniform {msd_u:.4f}")
    assert log["mean_J_last"] > log["mean_J_first"]
    assert msd1 > 1.1 * msd0
    assert abs(msd1 - msd2) < 0.05 * msd2
