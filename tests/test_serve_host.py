"""Host logic of the serving loop and its tuners (no GPU): the memory
estimate, the request distribution, the tuner's size classes and the bin-fit
rule, the stop test and Poisson arrivals."""
import numpy as np

from paper_2011_10214_gb300 import capi, serve
from paper_2011_10214_gb300 import workloads as wl


def test_size_classes_cover_the_distribution():
    rng = np.random.default_rng(5)
    cfgs = serve.request_distribution(rng, 400, big_fraction=0.05)
    classes = {serve.size_class(c) for c in cfgs}
    assert classes <= {(a, b) for a in (0, 1) for b in (0, 1, 2)}
    for c in cfgs:
        n, ppc = c["n"][0], c["species"][0]["ppc"]
        a, b = serve.size_class(c)
        assert a == (0 if n < 32 else 1)
        assert b == (0 if ppc <= 32 else 1 if ppc <= 48 else 2)


def test_bin_fit_rule():
    # edge 4 always fits the distribution's 16..64 ppc; edge 8 up to 51 ppc
    assert all(serve.fits_bin(p, 4) for p in range(1, 65))
    assert serve.fits_bin(51, 8) and not serve.fits_bin(52, 8)
    # the rule is the library's capacity: count + 25 % + 64 against 32767
    for p in (16, 40, 51, 52, 64):
        assert serve.fits_bin(p, 8) == (p * 512 * 1.25 + 64 <= 32767)


def test_memory_estimate_grows_with_size():
    small = wl.sphere_config(16, 2.0, 16, 500)
    big = wl.sphere_config(48, 8.0, 64, 500)
    a, b = serve.estimate_bytes(small, capi.MIXED), serve.estimate_bytes(big, capi.MIXED)
    assert 0 < a < b
    assert serve.estimate_bytes(big, capi.FP64) > b


def test_poisson_arrivals_are_increasing_and_bounded():
    rng = np.random.default_rng(9)
    t = serve.poisson_arrivals(rng, 20.0, 10.0)
    assert len(t) > 100 and all(0 < x <= 10.0 for x in t)
    assert all(b > a for a, b in zip(t, t[1:]))


def test_stop_rule():
    srv = object.__new__(serve.Server)
    srv.max_steps, srv.window, srv.rel = 500, 50, 0.01
    m = serve.Member(0, {}, 0.0, None, 0.0)
    m.steps = 60
    m.history = [(10, 1.0), (60, 1.005)]
    assert serve.Server._done(srv, m)            # < 1 % change over the window
    m.history = [(10, 1.0), (60, 1.05)]
    assert not serve.Server._done(srv, m)
    m.steps = 500
    assert serve.Server._done(srv, m)            # the step cap
