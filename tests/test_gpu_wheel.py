"""GPU parity of the Parisi-Rapuano wheel stream (Sec. 3.3, Eq. 5) on the
plain layout, through the C ABI against the CPU oracle, plus the
statistical cross-check the wheel is for: the same physics as the
counter-based stream.

Integer work, so bit-exact: spins after every sweep, E, M, F, Q, PT state.
Sizes cover L = 2 (one site per row and colour, every wheel advancing one
step a sweep), ragged sample counts, 2D and 3D, field models with empty
sites (which consume their wheel output all the same).
"""

import numpy as np
import pytest

from oracle import DIS_DAFF, DIS_EA, DIS_RFIM, HEATBATH, METROPOLIS, RNG_WHEEL, Oracle
from tests import pins

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000D00
NAMES = {DIS_EA: "pm_j", DIS_RFIM: "rfim", DIS_DAFF: "daff"}


def _pair(ianus, disorder=DIS_EA, dim=3, L=4, S=1, R=1, K=1, h=0.0, occ=1.0, seed=SEED):
    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed, layout="i8",
                        disorder=NAMES[disorder], field=h, occupation=occ, rng="wheel", series_capacity=4096)
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, n_temps=K, seed=seed, disorder=disorder,
                 field=h, occupation=occ, rng=RNG_WHEEL)
    return lat, orc


CASES = [(3, 2, 1, 1, 1), (3, 4, 3, 2, 1), (2, 4, 5, 1, 1), (3, 6, 7, 2, 2), (2, 8, 2, 2, 1), (3, 10, 2, 1, 1),
         (2, 2, 3, 2, 1)]


@pytest.mark.parametrize("disorder,h,occ", [(DIS_EA, 0.0, 1.0), (DIS_RFIM, 1.25, 1.0), (DIS_DAFF, 0.75, 0.7)])
@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("dim,L,S,R,K", CASES)
def test_wheel_sweep_bit_exact_every_sweep(ianus, disorder, h, occ, algo, dim, L, S, R, K):
    lat, orc = _pair(ianus, disorder, dim=dim, L=L, S=S, R=R, K=K, h=h, occ=occ, seed=SEED + 5 * L + S)
    beta = [0.7, 1.1][:K]
    for _ in range(5):
        lat.sweep(algo, beta, 1)
        orc.sweep(algo, beta, 1)
        assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


def test_wheel_series_graphs_and_checkpoint(ianus):
    lat, orc = _pair(ianus, dim=3, L=8, S=5, R=2)
    lat.sweep(HEATBATH, 0.9, 23, measure_every=5)
    orc.sweep(HEATBATH, 0.9, 23, measure_every=5)
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert list(sw) == list(swo) == [5, 10, 15, 20]
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)
    eager, _ = _pair(ianus, dim=3, L=8, S=5, R=2)
    eager.set_graphs(False)
    eager.sweep(HEATBATH, 0.9, 23, measure_every=5)
    assert np.array_equal(eager.spins(), lat.spins())
    # the checkpoint carries the wheels: the continuation is the same
    blob = lat.get_state()
    lat.sweep(METROPOLIS, 0.9, 9)
    other, _ = _pair(ianus, dim=3, L=8, S=5, R=2)
    other.set_state(blob)
    other.sweep(METROPOLIS, 0.9, 9)
    assert np.array_equal(other.spins(), lat.spins())


def test_wheel_parallel_tempering(ianus):
    """Sweeps draw from the wheels of the configurations, swaps from the PT
    stream; temperature labels move, wheels stay with their slots."""
    K = 4
    beta = [1.0 / (0.7 + 0.3 * k) for k in range(K)]
    lat, orc = _pair(ianus, dim=3, L=4, S=3, R=2, K=K)
    for _ in range(4):
        lat.sweep(METROPOLIS, beta, 5)
        lat.pt_swap()
        orc.sweep(METROPOLIS, beta, 5)
        orc.pt_swap(beta)
    assert np.array_equal(lat.spins(), orc.spins())
    sa, acc, steps = lat.pt_state()
    sao, acco, stepso = orc.pt_state()
    assert np.array_equal(sa, sao) and np.array_equal(acc, acco) and steps == stepso


def test_wheel_errors(ianus):
    with pytest.raises(ianus.IanusError) as e:
        ianus.Lattice(dim=3, L=4, layout="bits64", rng="wheel")
    assert e.value.status == ianus.EUNSUPPORTED
    with pytest.raises(ianus.IanusError):
        ianus.Lattice(model="potts", dim=3, L=4, rng="wheel")
    auto = ianus.Lattice(dim=3, L=4, n_samples=2, seed=4, rng="wheel")  # AUTO -> plain layout
    plain = ianus.Lattice(dim=3, L=4, n_samples=2, seed=4, rng="wheel", layout="i8")
    auto.sweep(HEATBATH, 0.8, 3)
    plain.sweep(HEATBATH, 0.8, 3)
    assert np.array_equal(auto.spins(), plain.spins())


@pytest.mark.parametrize("T", [2.0, 3.0])
def test_wheel_onsager_on_gpu(ianus, T):
    """The statistical cross-check at scale: 2D ferromagnet L=64, 64 samples,
    heat bath driven by the wheels, against Onsager's energy per site."""
    beta = 1.0 / T
    lat = ianus.Lattice(dim=2, L=64, n_samples=64, seed=SEED + 9, layout="i8", ferro=True, rng="wheel",
                        series_capacity=4096)
    if T < 2.27:
        lat.set_spins(np.ones((64, 1, 64 * 64), dtype=np.int8))
    lat.sweep(HEATBATH, beta, 500)
    lat.series(clear=True)
    lat.sweep(HEATBATH, beta, 2000, measure_every=2)
    _, E, _, _ = lat.series()
    e = E[:, :, 0, 0].astype(np.float64).mean(axis=1) / 4096.0
    mean, err = pins.batch_mean_error(e, nbatch=20)
    exact = pins.onsager_energy_per_site(beta)
    assert abs(mean - exact) < 4 * err + 2e-4, (mean, exact, err)


def test_wheel_and_philox_sample_the_same_distribution(ianus):
    """EA glass, 3D L=8, 128 samples, T = 2.0 (fast equilibration): on the
    same couplings, the per-sample mean energies of the two streams differ
    by thermal noise only (paired test over the samples)."""
    means = {}
    for rng in ("philox", "wheel"):
        lat = ianus.Lattice(dim=3, L=8, n_samples=128, seed=SEED + 10, layout="i8", rng=rng, series_capacity=4096)
        lat.sweep(HEATBATH, 0.5, 300)
        lat.series(clear=True)
        lat.sweep(HEATBATH, 0.5, 1000, measure_every=5)
        _, E, _, _ = lat.series()
        means[rng] = E[:, :, 0, 0].astype(np.float64).mean(axis=0) / 512.0
    d = means["philox"] - means["wheel"]
    assert abs(d.mean()) < 5 * d.std(ddof=1) / np.sqrt(len(d)), (d.mean(), d.std(ddof=1))
