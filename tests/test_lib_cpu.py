"""Host-side checks of the CUDA library that need no GPU: it builds, loads, exports
every entry point declared in include/wavprop.h, and its host-only arithmetic
(FD weights, CFL limit, memory estimate) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1808_01995_gb300 import build as B
from paper_1808_01995_gb300 import wavprop as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return W.lib()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"\b(wp_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert {"wp_forward", "wp_adjoint", "wp_gradient", "wp_forward_dev"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert missing == []
    assert set(W.EXPORTED) <= names


@pytest.mark.parametrize("k", range(2, 17, 2))
def test_fd_weights_match_oracle(lib, k):
    assert np.allclose(W.wp_fd_weights(k), O.fd_weights(k), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("ndim,k", [(2, 4), (3, 8), (3, 16), (2, 2)])
def test_cfl_matches_oracle(lib, ndim, k):
    h = (10.0, 12.0, 9.0)[:ndim]
    g = W.Grid((20,) * ndim, h, (0.0,) * ndim, k)
    assert abs(W.wp_cfl_dt(g, 3700.0) / O.cfl_dt(h, k, 3700.0) - 1) < 1e-13


def test_invalid_arguments_are_rejected_on_the_host(lib):
    with pytest.raises(W.WpError) as e:
        W.wp_fd_weights(5)
    assert e.value.status == W.WP_EINVAL
    with pytest.raises(W.WpError) as e:
        W.wp_cfl_dt(W.Grid((1, 5), (1.0, 1.0), (0.0, 0.0), 4), 1.0)
    assert e.value.status == W.WP_EINVAL
    with pytest.raises(W.WpError):
        W.wp_cfl_dt(W.Grid((5, 5), (1.0, 1.0), (0.0, 0.0), 18), 1.0)


def test_memory_estimate_grows_with_snapshots(lib):
    g = W.Grid((64, 64, 64), (10.0,) * 3, (0.0,) * 3, 8, 1e-3, 100)
    f = W.wp_estimate_bytes(g, 1, 100, 0)
    g1 = W.wp_estimate_bytes(g, 1, 100, 1, 10)
    g2 = W.wp_estimate_bytes(g, 1, 100, 1, 5)
    field = 64 * 64 * 64 * 4
    assert f >= 4 * field and g1 > f + 20 * field and g2 > g1
