"""Host-only entry points of the C ABI, on the CPU: the search grid, the
analytic choice (Eqs. 2-3 with the GB300 rates), the default configuration's
method switch and the selector's parameter layout.  None of them touches the
GPU."""
import ctypes
import os

import numpy as np
import pytest

from oracle import selector as so


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_06872_gb300 import binding as b
    b.load()
    return b


def test_grid_points_follow_the_documented_table(binding):
    n, m = 1 << 24, 16 << 24
    g = [binding.grid_config(i, n, m).as_dict() for i in range(binding.TUNE_GRID)]
    assert g[0]["method"] == 0 and g[0]["hdv_k"] == 0 and g[0]["flags"] & binding.FLAG_AGGREGATE
    assert g[1]["method"] == 0 and g[1]["hdv_k"] == 512 and (1 << g[1]["table_log2"]) >= 2 * 512
    radix = [(g[i]["method"], g[i]["radix_tile"], g[i]["ctas_per_sm"], g[i]["radix_digit_bits"]) for i in range(2, 12)]
    assert radix == [(1, 0, 4, 8), (1, 0, 4, 7), (1, 0, 4, 6), (1, 4096, 2, 8), (1, 4096, 2, 7), (1, 4096, 3, 6),
                     (1, 2048, 4, 8), (1, 2048, 4, 7), (1, 2048, 6, 8), (1, 2048, 6, 6)]
    assert all(g[i]["hdv_k"] == 0 for i in range(2, 12))
    # an HDV count above n / 2 becomes 0 (the point equals Atomic GT)
    assert binding.grid_config(1, 1000, 50000).hdv_k == 0
    with pytest.raises(binding.GtError) as ei:
        binding.grid_config(binding.TUNE_GRID, n, m)
    assert ei.value.code == 1


def test_default_config_switches_method_at_4m_edges(binding):
    assert binding.default_config(1 << 20, (1 << 22) - 1).method == 0
    assert binding.default_config(1 << 20, 1 << 22).method == 1
    assert binding.default_config(1 << 28, 1 << 32).method == 1


def _features(coverage, same_line=0.0, weighted=True):
    f = np.zeros(so.N_FEATURES, dtype=np.float32)
    f[36] = coverage
    f[39] = same_line
    f[40] = 1.0 if weighted else 0.0
    return f


def test_analytic_choice(binding):
    # far beyond L2 (scale 28): at the coverage R-MAT gives (a few % to ~40 %) streaming wins
    for c in (0.0, 0.25, 0.5):
        assert binding.analytic_index(_features(c), 1 << 28, 1 << 32) == 2
    # an L2-resident graph: the HDV split pays once the HDVs cover most edges ...
    assert binding.analytic_index(_features(0.9), 1000, 20000) == 1
    # ... and with no coverage its hash probes only add to Atomic GT, so the choice leaves HLH
    assert binding.analytic_index(_features(0.0), 1000, 20000) != 1
    # more coverage never moves the choice from HLH back to another method
    picks = [binding.analytic_index(_features(c), 5000, 100000) for c in np.linspace(0, 1, 21)]
    assert picks[-1] == 1 and picks[0] != 1
    first = picks.index(1)
    assert all(p == 1 for p in picks[first:])
    lib = binding.load()
    idx = ctypes.c_uint32()
    assert lib.gt_tune_analytic(None, 10, 10, ctypes.byref(idx)) == 1


def test_selector_parameter_layout_matches_the_oracle(binding):
    assert binding.load().gt_selector_param_count() == so.layout()["total"] == 7792
    assert binding.N_FEATURES == so.N_FEATURES and binding.TUNE_GRID == so.GRID
    p = np.fromfile(os.path.join(os.path.dirname(binding.__file__), "selector_params.f32"), dtype="<f4")
    assert p.size == so.layout()["total"]
    o, k = so.layout()["sd"]
    assert np.all(p[o:o + k] > 0)  # standardisation scales are positive
    lo, hi = so.layout()["lo"][0], so.layout()["hi"][0]
    assert np.all(p[lo:lo + so.N_FEATURES] <= p[hi:hi + so.N_FEATURES])  # trained feature range
