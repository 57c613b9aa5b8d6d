"""ianus_prepare_sweep: the kernel a sweep would specialise for its
temperature, compiled ahead (on worker threads) without touching the
lattice, and a switch from the precompiled kernel (variant 1) to the
specialised one in the middle of a run.  Trajectories are compared bit for
bit with the oracle: the switch must not change a single spin."""

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import HEATBATH, METROPOLIS, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000000 + 700


def _series_equal(lat, orc, R):
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    same = np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)
    return same and (R < 2 or np.array_equal(Q, Qo))


def test_prepare_reports_ready_and_leaves_the_lattice_alone(ianus):
    lat = ianus.Lattice(dim=3, L=8, n_samples=70, n_replicas=2, seed=SEED, layout="bits64")
    before = lat.get_state()
    assert lat.prepare_sweep(HEATBATH, 0.913, 0)
    assert lat.prepare_sweep(METROPOLIS, 0.913, 24)
    assert lat.prepare_sweep(HEATBATH, 0.913, 26)     # the persistent form
    assert not lat.prepare_sweep(HEATBATH, 0.913, 1)  # variant 1 specialises nothing
    assert lat.get_state() == before
    assert lat.sweeps == 0


def test_prepare_on_lattices_without_a_specialised_kernel(ianus):
    plain = ianus.Lattice(dim=3, L=8, n_samples=4, n_replicas=1, seed=SEED, layout="i8")
    assert not plain.prepare_sweep(HEATBATH, 1.0, 0)
    pt = ianus.Lattice(dim=3, L=8, n_samples=64, n_replicas=2, n_temps=2, seed=SEED, layout="bits64")
    assert not pt.prepare_sweep(HEATBATH, [0.9, 1.0], 0)


def test_prepare_validation(ianus):
    lat = ianus.Lattice(dim=3, L=8, n_samples=64, n_replicas=1, seed=SEED, layout="bits64")
    for args in ((HEATBATH, 1.0, 28), (HEATBATH, 1.0, -1), (7, 1.0, 0), (HEATBATH, float("nan"), 0),
                 (HEATBATH, -0.5, 0)):
        with pytest.raises(ianus.IanusError) as e:
            lat.prepare_sweep(*args)
        assert e.value.status == ianus.EINVAL


@pytest.mark.parametrize("variant_after", [0, 22, 25])
def test_switch_from_precompiled_to_prepared_kernel_mid_run(ianus, variant_after):
    """Five sweeps on the precompiled kernel, then the prepared kernel: the
    series and the final spins equal the oracle's uninterrupted run."""
    beta = 0.871
    lat = ianus.Lattice(dim=3, L=12, n_samples=100, n_replicas=2, seed=SEED + 1, layout="bits64")
    lat.set_variant(1)
    lat.sweep(HEATBATH, beta, 5, measure_every=5)
    assert lat.prepare_sweep(HEATBATH, beta, variant_after)
    lat.set_variant(variant_after)
    lat.sweep(HEATBATH, beta, 7, measure_every=1)
    orc = Oracle(dim=3, L=12, sample_ids=list(range(100)), n_replicas=2, seed=SEED + 1)
    orc.sweep(HEATBATH, beta, 5, measure_every=5, nthreads=8)
    orc.sweep(HEATBATH, beta, 7, measure_every=1, nthreads=8)
    assert np.array_equal(lat.spins(), orc.spins())
    assert _series_equal(lat, orc, 2)


def test_concurrent_prepares_while_sweeping(ianus):
    """Eight worker threads compile kernels for different temperatures and
    shapes (two threads on each kernel) while the main thread sweeps another
    lattice; afterwards every prepared kernel runs bit-exact."""
    cases = [(3, 8, 64, 2, HEATBATH, 0.5 + 0.137 * k) for k in range(3)] + \
            [(2, 16, 65, 1, METROPOLIS, 0.6 + 0.091 * k) for k in range(1)]
    lats = [ianus.Lattice(dim=d, L=L, n_samples=S, n_replicas=R, seed=SEED + 10 + i, layout="bits64")
            for i, (d, L, S, R, _, _) in enumerate(cases)]
    busy = ianus.Lattice(dim=3, L=16, n_samples=128, n_replicas=2, seed=SEED + 20, layout="bits64")
    busy.set_variant(1)
    with ThreadPoolExecutor(max_workers=8) as pool:
        futs = [pool.submit(lat.prepare_sweep, c[4], c[5], 0) for lat, c in zip(lats, cases) for _ in range(2)]
        busy.sweep(HEATBATH, 1.0, 30)
        assert all(f.result() for f in futs)
    busy.synchronize()
    for lat, (d, L, S, R, algo, beta), i in zip(lats, cases, range(len(cases))):
        lat.sweep(algo, beta, 6, measure_every=3)
        orc = Oracle(dim=d, L=L, sample_ids=list(range(S)), n_replicas=R, seed=SEED + 10 + i)
        orc.sweep(algo, beta, 6, measure_every=3, nthreads=8)
        assert np.array_equal(lat.spins(), orc.spins())
        assert _series_equal(lat, orc, R)
