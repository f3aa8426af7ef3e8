"""The device watchdog (opts.watchdog_every, sim_watchdog): its energy proxy
against the definition summed in NumPy from the fields the handle returns,
silence on a stable run, and a trip on a run whose time step is past the
scheme's stability limit, on growth alone (every value still finite)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _short_pulse(cfl=0.5, f0=5e5):
    """The 70x16x320 cased well with a short source pulse, so that the
    source is silent after a few dozen steps (the wavelet table covers
    8 / f0)."""
    sc = W.config1(steps=400)
    return dataclasses.replace(sc, source=dataclasses.replace(sc.source, f0=f0), cfl=cfl)


def proxy(sim, med):
    """1/2 sum [rho |v|^2 + (s_rr^2 + s_pp^2 + s_zz^2 + 2 (s_rp^2 + s_pz^2 +
    s_rz^2)) / (lambda + 2 mu)] over every cell, each with its own material."""
    f = {n: sim.field(n).astype(np.float64) for n in oracle.FIELDS}
    rho = med.rho[med.cell_id]
    M = np.float32(med.rho * med.vp ** 2)[med.cell_id].astype(np.float64)  # stored as FP32
    v2 = f["vr"] ** 2 + f["vp"] ** 2 + f["vz"] ** 2
    s2 = f["srr"] ** 2 + f["spp"] ** 2 + f["szz"] ** 2 + 2 * (f["srp"] ** 2 + f["spz"] ** 2 + f["srz"] ** 2)
    return 0.5 * float(np.sum(np.float32(rho).astype(np.float64) * v2 + s2 / M))


@pytest.mark.parametrize("storage,kernel", [("f32", "auto"), ("f16", "auto"), ("f32", "fused")])
def test_watchdog_proxy_equals_its_definition(storage, kernel):
    from paper_2302_13907_gb300.binding import Simulation
    sc = W.config1(steps=300)
    with Simulation(sc, storage=storage, kernel=kernel, watchdog_every=50, max_steps=300) as s:
        s.step(250)
        e, ref, n = s.watchdog()
        assert n == 250
        want = proxy(s, sc.medium)
        assert want > 0
        assert e == pytest.approx(want, rel=1e-5)
        # the 10 kHz pulse lasts 8 / f0 = 2680 steps here: no reference yet
        assert ref == 0.0
        assert s.sync() is None


def test_watchdog_is_silent_on_a_stable_run():
    """A 40 kHz pulse (7.5 cells per wavelength in the liquid, so the energy
    travels; the wavelet table ends after 670 steps) over 2400 steps, long
    enough for the waves to reach the radial PML (about 400 steps) and the
    lower z end (about 700 after the pulse), with the PML and with rigid walls:
    no trip; with rigid walls (nothing leaves) the proxy stays within a small
    factor of its reference, and with the PML it ends lower (absorbed)."""
    from paper_2302_13907_gb300.binding import Simulation
    final = {}
    for pml_on in (True, False):
        sc = _short_pulse(f0=4e4)
        with Simulation(sc, watchdog_every=40, pml_on=pml_on, max_steps=2400) as s:
            hist = []
            for _ in range(60):
                s.step(40)
                hist.append(s.watchdog())
            s.sync()
            ref = hist[-1][1]
            assert ref > 0, pml_on
            after = [e for e, r, n in hist if r > 0]
            assert all(np.isfinite(after))
            print(f"pml_on={pml_on}: reference {ref:.4g}, later proxies {min(after) / ref:.3f} .. "
                  f"{max(after) / ref:.3f} of it, last {after[-1] / ref:.3f}")
            assert max(after) <= 5 * ref, pml_on
            if not pml_on:
                assert min(after) >= 0.1 * ref
            final[pml_on] = after[-1]
    assert final[True] < final[False], final


def test_watchdog_trips_on_growth_past_the_stability_limit():
    """CFL 1.4 (the scheme's limit on this grid is about 1.07, from the power
    iteration of the oracle's operator, and the steel casing sets it): the
    grid-scale modes of the casing grow about 4.7x per step once the wave from
    the axis reaches it (0.1 m at 1500 m/s, about 80 steps), long after the
    source fell silent (21 steps).  With a check after every step the watchdog
    trips on growth while every value is still finite."""
    from paper_2302_13907_gb300.binding import SIM_EUNSTABLE, SimError, Simulation
    sc = _short_pulse(cfl=1.4)
    with Simulation(sc, watchdog_every=1, max_steps=250, graph_chunk=-1) as s:
        tripped = None
        for n in range(1, 240):
            s.step(1)
            try:
                s.sync()
            except SimError as ex:
                tripped = (n, ex)
                break
        assert tripped is not None
        n, ex = tripped
        assert ex.code == SIM_EUNSTABLE and "watchdog" in str(ex), ex
        e, ref, step = s.watchdog()
        assert step == n and ref > 0 and np.isfinite(e) and e > 100 * ref
        print(f"tripped at step {n}: proxy {e:.3g} = {e / ref:.3g} x the reference")
        assert all(np.isfinite(s.field(f)).all() for f in oracle.FIELDS)


def test_watchdog_off_by_default_and_validated():
    from paper_2302_13907_gb300.binding import SIM_EINVAL, SimError, Simulation
    sc = W.config1(steps=10)
    with Simulation(sc) as s:
        with pytest.raises(SimError) as ei:
            s.watchdog()
        assert ei.value.code == SIM_EINVAL
