"""The seeded workloads have the sizes and layouts the benchmark reports: HERA-like hexagons
of 14.6 m spacing at latitude -30.72 deg (Sec. 3.1), a 1 h drift scan, the stripe grid, the
mode and gain-parameter counts.  Everything here is counted from the generated arrays."""
import itertools
import math

import numpy as np
import pytest

from paper_2504_07090_gb300 import synth


@pytest.mark.parametrize("name,n_ant,n_freq,band,n_lst,n_pix,n_modes", [
    ("cfg0", 7, 16, (150e6, 160e6), 20, 3072, 512),
    ("cfg1", 37, 64, (140e6, 160e6), 60, 24576, 16384),
    ("cfg4", 127, 128, (120e6, 180e6), 120, 98304, 65536),
])
def test_named_workload_sizes(name, n_ant, n_freq, band, n_lst, n_pix, n_modes):
    p = synth.config(name)
    assert p.n_ant == n_ant and p.n_bl == n_ant * (n_ant - 1) // 2
    assert p.n_freq == n_freq and p.freq_hz[0] == band[0] and p.freq_hz[-1] == band[1]
    assert p.n_lst == n_lst and p.n_pix == n_pix and p.n_modes == n_modes
    assert p.n_params == n_freq * n_modes + 2 * n_ant * 4          # 4 complex gain modes per antenna
    # 1 h of LST at a uniform cadence, centred in an RA stripe that covers it with margin
    step = np.diff(p.lst_rad)
    np.testing.assert_allclose(step, 15.0 * math.pi / 180.0 / n_lst, rtol=1e-12)
    assert p.ra_min < p.lst_rad[0] and p.lst_rad[-1] < p.ra_max
    # the stripe: declination band of +-10 deg about the array latitude
    np.testing.assert_allclose(0.5 * (p.dec_min + p.dec_max), p.lat_rad, atol=1e-15)
    np.testing.assert_allclose(p.lat_rad, -30.72 * math.pi / 180.0, atol=1e-15)
    np.testing.assert_allclose(p.dec_max - p.dec_min, 20.0 * math.pi / 180.0, atol=1e-15)


def test_cfg1_parameter_count():
    assert synth.config("cfg1").n_params == 1_048_872


@pytest.mark.parametrize("side,n_ant", [(2, 7), (3, 19), (4, 37), (7, 127)])
def test_hexagon_spacing_and_count(side, n_ant):
    ant = synth.hex_array(side)
    assert ant.shape == (n_ant, 3) and np.all(ant[:, 2] == 0.0)
    d = [np.linalg.norm(a - b) for a, b in itertools.combinations(ant, 2)]
    assert abs(min(d) - 14.6) < 1e-12                                 # nearest neighbours
    # every antenna of the interior has six neighbours at 14.6 m, the centre included
    centre = np.argmin(np.linalg.norm(ant[:, :2], axis=1))
    near = np.sum(np.abs(np.linalg.norm(ant - ant[centre], axis=1) - 14.6) < 1e-9)
    assert near == 6


def test_batch_problems_are_uneven_and_seeded():
    a = synth.batch_problems()
    b = synth.batch_problems()
    assert len(a) == 64
    assert [p.n_params for p in a] == [p.n_params for p in b]           # reproducible
    assert {p.n_ant for p in a} == {7, 19, 37}
    assert {p.n_freq for p in a} == {16, 32, 64}
    assert all(p.n_lst == 20 for p in a)
    assert min(p.n_modes for p in a) == 512 and max(p.n_modes for p in a) == 16384
