"""The dynamic test of Sec. 4.2 on the oracle (no GPU): an isothermal
(T = 1e4 K), homogeneous sphere of column N_HI = 2e20 cm^-2 in Hubble
expansion v = v_max r / R.  The paper: raising v_max suppresses the blue peak
until it is gone by v_max ~ 200 km/s; the red peak first moves away from line
centre, and past a critical v_max comes back towards it, since the velocity
gradient eases escape.  The static sphere is symmetric."""
import numpy as np

from paper_1409_4480_gb300 import synth as S

TAU0 = 2e20 * 5.898e-14        # N_HI sigma_0 at T = 1e4 K (Sec. 2)


def _run(O, v, n):
    g = S.sphere(24, 1e4, TAU0, v_max_kms=v)
    spec = S.RunSpec(n_packets=n, seed=40, albedo=0.0, spec_units=1, spec_lo=-1500.0, spec_hi=1500.0,
                     spec_nbins=150)
    r = O.run(g, spec)
    assert r["n_escaped"] == n
    s = r["spec"].astype(float)
    centres = np.linspace(-1490.0, 1490.0, 150)
    red = s[75:]
    # blue = Delta v < 0, escapes below the range included (red above it)
    blue = (s[:75].sum() + r["spec_under"]) / n
    return blue, centres[75 + np.argmax(np.convolve(red, np.ones(5) / 5, "same"))]


def test_expanding_sphere_blue_peak_and_red_peak(O):
    out = {v: _run(O, v, 600) for v in (0.0, 20.0, 50.0, 200.0, 2000.0)}
    blue = [out[v][0] for v in (0.0, 20.0, 50.0, 200.0)]
    print({v: (round(b, 3), r) for v, (b, r) in out.items()})
    assert abs(blue[0] - 0.5) < 0.07                       # static: symmetric
    assert blue[0] > blue[1] > blue[2] >= blue[3]         # the blue peak fades ...
    assert blue[3] < 0.01                                 # ... and is gone by 200 km/s
    assert out[200.0][1] > out[0.0][1]                    # the red peak moves out ...
    assert out[2000.0][1] < out[200.0][1]                 # ... and back past a critical v_max
