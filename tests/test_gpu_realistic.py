"""The paper's realistic well (Sec. 6) on the GPU: parity with the oracle on
a section around a collar, and the paper's observation that a torsion source
on the casing wall launches a wave that runs along that casing at the
steel's shear speed (3220 m/s), through its couplings, while the liquid
around it and everything beyond stays at rest."""
import numpy as np
import pytest

import oracle
from paper_2302_13907_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_realistic_section_around_a_collar_matches_the_oracle():
    sc = W.realistic_well_section(z0=11.6, length=0.8, nth=8, nr=64, pml_r=8, pml_z=8, f0=20e3,
                                  source_depth=11.8, steps=1000)
    from paper_2302_13907_gb300.binding import Simulation
    o = oracle.Oracle(sc)
    o.step(sc.steps)
    with Simulation(sc) as s:
        s.step(sc.steps)
        scale = {k: max(np.abs(o.field(n)).max() for n in oracle.FIELDS if n[0] == k) for k in "vs"}
        assert scale["v"] > 0 and scale["s"] > 0
        for n in oracle.FIELDS:
            a, b = s.field(n), o.field(n)
            assert np.abs(a - b).max() <= 2e-5 * scale[n[0]], (n, np.abs(a - b).max() / scale[n[0]])


def test_torsion_wave_runs_along_the_casing_at_the_steel_shear_speed():
    z0, src = 100.0, 103.0
    sc = W.realistic_well_section(z0=z0, length=12.0, nth=8, nr=64, f0=8e3, source_depth=src, steps=20000)
    from paper_2302_13907_gb300.binding import Simulation
    g = sc.medium.grid
    rc = g.r_centre()
    row = int(np.argmin(np.abs(rc - (0.1778 / 2 - 0.00919 / 2))))  # middle of the target casing wall
    outside = rc > 0.1945 / 2  # annulus liquid, exterior casing, rock
    k = [int(round((src + d - z0) / g.dz)) + g.pml_z for d in (2.0, 6.0)]  # the collar at 108 m lies between
    every = 20
    with Simulation(sc, graph_chunk=every) as s:
        dt = s.dt
        n = int((2.0 / 8e3 + 6.5 / 3220.0 + 2.0 / 8e3) / dt / every) + 1
        hist, ann = [], 0.0
        for _ in range(n):
            s.step(every)
            vp = s.field("vp")
            hist.append([vp[:, row, kk].mean() for kk in k])
            ann = max(ann, float(np.abs(vp[:, outside, :]).max()))
    h = np.array(hist)
    peak = np.abs(h).max()
    assert peak > 0 and ann == 0.0  # no azimuthal motion outside the casing at all
    a, b = h[:, 0] - h[:, 0].mean(), h[:, 1] - h[:, 1].mean()
    xc = np.correlate(b, a, mode="full")
    m = int(np.argmax(xc))
    y0, y1, y2 = xc[m - 1], xc[m], xc[m + 1]
    lag = (m - (len(a) - 1)) + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    speed = 4.0 / (lag * every * dt)
    print(f"torsion wave speed along the casing: {speed:.1f} m/s")
    import json
    import os
    paper = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_realistic_well.json")))
    c = paper["torsion_wave_speed_m_s"]  # Sec. 6
    assert abs(speed - c) < 0.01 * c, speed
