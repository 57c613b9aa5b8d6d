"""Pins of the oracle's parallel-tempering bookkeeping (Sec. 2.2 names
parallel tempering; the swap rule is the standard min(1, exp(dbeta * dE))).

Two mappings carry the labels once configurations have been exchanged, and
each is checked here against something fixed outside the oracle:

* a sweep gives every configuration the beta of the temperature it now
  holds.  With beta = 0 a Metropolis sweep negates every spin (the threshold
  2^32 lies above every random), and with beta = 40 no move that raises the
  energy is accepted (floor(2^32 exp(-160)) = 0).  So after a swap the
  configuration at the beta = 0 label must come back exactly negated, and the
  ones at beta = 40 must not rise in energy;
* measurement rows are indexed by temperature: E, M and Q of row (sample, k)
  are those of the configurations that hold temperature k, evaluated here in
  numpy (E by the bond sum of Eq. (2), M and Q from their definitions) on the
  read-back spins gathered through the oracle's slot map.

With these betas every swap decision is deterministic: the random threshold
is 0 (never) or the rule's "always" branch, so the expected exchanges follow
from the energies alone.
"""

import numpy as np

from oracle import METROPOLIS, Oracle
from tests import pins

SEED = 0x0704357300000000 + 40


def _energy(config, J, L, D):
    return pins.ising_energy(config, J, L, D)


def _random_pair_with_gap(rng, J, L, D, N):
    """Two random configurations with E(hi) > E(lo)."""
    while True:
        a = rng.choice([-1, 1], size=N).astype(np.int8)
        b = rng.choice([-1, 1], size=N).astype(np.int8)
        ea, eb = _energy(a, J, L, D), _energy(b, J, L, D)
        if ea != eb:
            return (a, b) if ea < eb else (b, a)


def test_pt_sweep_uses_the_beta_of_the_temperature_label_k2():
    """K = 2, beta = (0, 40), R = 2.  Pair (0, 1) has dbeta = -40 < 0, so it
    exchanges iff E(config at 1) >= E(config at 0), and never otherwise
    (threshold 0).  Each round places a low and a high energy configuration
    so that a chosen chain exchanges and the other does not, then checks the
    exchange and the next sweep through the labels."""
    L, D = 4, 3
    N = L ** D
    beta = [0.0, 40.0]
    ids = [0, 70]
    R, K = 2, 2
    o = Oracle(dim=D, L=L, sample_ids=ids, n_replicas=R, n_temps=K, seed=SEED)
    J = o.couplings()
    rng = np.random.default_rng(5)
    plans = [(True, False), (False, True), (True, True), (True, False), (False, False), (False, True)]
    saw_permuted = False
    for want in plans:
        slot_at, _, _ = o.pt_state()
        sp = o.spins()
        for si in range(len(ids)):
            for a in range(R):
                lo, hi = _random_pair_with_gap(rng, J[si], L, D, N)
                # exchange wanted: the higher energy at the cold label (k = 1)
                at0, at1 = (lo, hi) if want[a] else (hi, lo)
                sp[si, slot_at[si, a, 0] * R + a] = at0
                sp[si, slot_at[si, a, 1] * R + a] = at1
        o.set_spins(sp)
        o.pt_swap(beta)
        after, _, _ = o.pt_state()
        for si in range(len(ids)):
            for a in range(R):
                expect = slot_at[si, a, ::-1] if want[a] else slot_at[si, a]
                assert np.array_equal(after[si, a], expect), (si, a, want)
        saw_permuted |= bool(np.any(after[:, :, 0] != 0))
        before = o.spins()
        o.sweep(METROPOLIS, beta, 1)
        now = o.spins()
        for si in range(len(ids)):
            for a in range(R):
                hot = after[si, a, 0] * R + a
                cold = after[si, a, 1] * R + a
                assert np.array_equal(now[si, hot], -before[si, hot]), (si, a)
                assert _energy(now[si, cold], J[si], L, D) <= _energy(before[si, cold], J[si], L, D)
                assert not np.array_equal(now[si, cold], -before[si, cold])
    assert saw_permuted


def test_pt_sweep_uses_the_beta_of_the_temperature_label_k3():
    """K = 3, beta = (0, 40, 40): pair (1, 2) has dbeta = 0 and always
    exchanges, so after a swap step a chain holds (B, C, A) if pair (0, 1)
    exchanged and (A, C, B) otherwise.  The configuration at label 0 must be
    negated by the next sweep; those at labels 1 and 2 must not rise."""
    L, D = 4, 3
    N = L ** D
    beta = [0.0, 40.0, 40.0]
    R, K = 2, 3
    o = Oracle(dim=D, L=L, sample_ids=[3], n_replicas=R, n_temps=K, seed=SEED + 1)
    J = o.couplings()
    rng = np.random.default_rng(6)
    for want in [(True, False), (False, True), (True, True), (False, False)]:
        slot_at, _, _ = o.pt_state()
        sp = o.spins()
        for a in range(R):
            lo, hi = _random_pair_with_gap(rng, J[0], L, D, N)
            at0, at1 = (lo, hi) if want[a] else (hi, lo)
            sp[0, slot_at[0, a, 0] * R + a] = at0
            sp[0, slot_at[0, a, 1] * R + a] = at1
        o.set_spins(sp)
        o.pt_swap(beta)
        after, _, _ = o.pt_state()
        for a in range(R):
            A, B, C = slot_at[0, a]
            expect = [B, C, A] if want[a] else [A, C, B]
            assert list(after[0, a]) == expect, (a, want)
        before = o.spins()
        o.sweep(METROPOLIS, beta, 1)
        now = o.spins()
        for a in range(R):
            hot = after[0, a, 0] * R + a
            assert np.array_equal(now[0, hot], -before[0, hot])
            for k in (1, 2):
                c = after[0, a, k] * R + a
                assert _energy(now[0, c], J[0], L, D) <= _energy(before[0, c], J[0], L, D)


def _rows_from_definitions(o, L, D):
    """E [S,K,R], M [S,K,R], Q [S,K] of the configurations holding each
    temperature, from the read-back spins and couplings."""
    sp = o.spins()
    J = o.couplings()
    slot_at, _, _ = o.pt_state()
    S, R, K = slot_at.shape
    E = np.zeros((S, K, R), dtype=np.int64)
    M = np.zeros((S, K, R), dtype=np.int64)
    Q = np.zeros((S, K), dtype=np.int64)
    for s in range(S):
        for k in range(K):
            conf = [sp[s, slot_at[s, a, k] * R + a].astype(np.int64) for a in range(R)]
            for a in range(R):
                E[s, k, a] = _energy(conf[a], J[s], L, D)
                M[s, k, a] = int(conf[a].sum())
            Q[s, k] = int((conf[0] * conf[1]).sum())
    return E, M, Q, slot_at


def test_pt_measurement_rows_are_indexed_by_temperature():
    """K = 4 close temperatures, R = 2: many exchanges, different in the two
    replicas' chains.  After every swap step, and in the series rows written
    after the following sweeps, the rows by temperature equal the definitions
    evaluated on the configurations that hold each temperature."""
    L, D = 4, 3
    beta = [0.50, 0.48, 0.46, 0.44]
    o = Oracle(dim=D, L=L, sample_ids=[0, 5, 70], n_replicas=2, n_temps=4, seed=SEED + 2)
    permuted = differ = 0
    for step in range(12):
        o.sweep(METROPOLIS, beta, 2, measure_every=2)
        o.pt_swap(beta)
        E, M, Q = o.measure()
        Ed, Md, Qd, slot_at = _rows_from_definitions(o, L, D)
        assert np.array_equal(E, Ed) and np.array_equal(M, Md) and np.array_equal(Q, Qd), step
        ident = np.arange(4)
        permuted += int(np.sum(np.any(slot_at != ident, axis=2)))
        differ += int(np.sum(np.any(slot_at[:, 0] != slot_at[:, 1], axis=1)))
        # series rows written after sweeps under this slot map
        o.clear_series()
        o.sweep(METROPOLIS, beta, 2, measure_every=1)
        _, Es, Ms, Qs = o.series()
        Ed, Md, Qd, _ = _rows_from_definitions(o, L, D)
        assert np.array_equal(Es[-1], Ed) and np.array_equal(Ms[-1], Md) and np.array_equal(Qs[-1], Qd), step
    # the check means something only once labels have moved, differently per replica
    assert permuted >= 10 and differ >= 5, (permuted, differ)
