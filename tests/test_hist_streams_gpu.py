"""Histogram streams: sorted points, intervals and records (Eq. 4), each against the FP64 oracle.

The interval stream sums each stretch of one bin along the gathered axis as a
difference of prefix sums of the factor tile; the record stream does the same
for up to eight consecutive bins of one line at once (one prefix sum more
than the bins present); the point
stream adds every point.  Each is forced in turn on every case and must meet
the histogram tolerance (1e-6 absolute per bin).  The run, interval and record
counts the device reports are checked exactly against counts from its bins.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1908_11246_gb300 import inputs as I
from tests import helpers as Hp

pytestmark = pytest.mark.gpu

MAX_PART_ROWS = 392


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_1908_11246_gb300 import build
    build.build()


def _cases():
    return [
        I.config("c2", "small"), I.config("c3", "small"), I.config("c4", "small"),
        I.random_problem(301, ndim=2), I.random_problem(302, ndim=3), I.random_problem(303, ndim=2),
        I.Problem("ipsa_ex", (300, 120), (-5.0, -1.5), (5.0, 1.5), I.MODEL_IPSA_EXAMPLE_2D, (),
                  I.random_densities(np.random.default_rng(31), 200, (-5.0, -1.5), (5.0, 1.5),
                                     sig=(0.05, 0.8)), 1000),
        # gathered axis of 900 rows: three parts of 300 rows
        I.Problem("parts3", (900, 70), (-3.0, -2.0), (3.0, 2.0), I.MODEL_SIN_SIN2_2D, (1.0, 7.0),
                  I.random_densities(np.random.default_rng(32), 300, (-3.0, -2.0), (3.0, 2.0),
                                     sig=(0.02, 0.8)), 64),
    ]


CASES = _cases()


def layout_counts(bins_nd, B, layout):
    """Runs and intervals of a layout, counted from the bins on the host.

    layout 0 gathers the last axis, layout 1 (2-D) axis 0.  The gathered axis
    is cut into parts of ceil(n / P) rows, P = ceil(n / 392) (one part when
    P * B > 32768); runs are maximal stretches of one (part, bin) key and one
    rest index in the stable sort by key, intervals the stretches of a run
    whose gathered rows are consecutive.
    """
    b = bins_nd if layout == 0 else bins_nd.T
    n_last = b.shape[-1]
    b = b.reshape(-1, n_last)
    P = -(-n_last // MAX_PART_ROWS)
    if P * B > 32768:
        P = 1
    pr = -(-n_last // P)
    R = b.shape[0]
    a = np.tile(np.arange(n_last), R)
    rest = np.repeat(np.arange(R), n_last)
    key = (a // pr) * B + b.ravel()
    order = np.argsort(key, kind="stable")
    k, r, aa = key[order], rest[order], a[order]
    new_run = np.ones(k.size, bool)
    new_run[1:] = (k[1:] != k[:-1]) | (r[1:] != r[:-1])
    new_iv = new_run.copy()
    new_iv[1:] |= aa[1:] != aa[:-1] + 1
    return int(new_run.sum()), int(new_iv.sum()), record_count(b.ravel(), n_last, pr, B)


def record_count(bins_lines, n_last, pr, B, G=8):
    """Records of the record stream: the intervals of every line in line order
    (maximal stretches of one (part, bin) key), grouped while the line, the
    part and the group of G bins stay the same and the bin steps keep their
    sign (a step whose sign differs from the step before starts a record)."""
    a = np.tile(np.arange(n_last), bins_lines.size // n_last)
    key = (a // pr) * B + bins_lines
    start = np.ones(key.size, bool)
    start[1:] = (a[1:] == 0) | (key[1:] != key[:-1])
    k = key[start]
    line = (np.flatnonzero(start) // n_last)
    part, grp = k // B, (k % B) // G
    same = np.zeros(k.size, bool)
    same[1:] = (line[1:] == line[:-1]) & (part[1:] == part[:-1]) & (grp[1:] == grp[:-1])
    rec = ~same
    up = np.zeros(k.size, bool)
    up[1:] = k[1:] > k[:-1]
    turn = np.zeros(k.size, bool)
    turn[2:] = same[2:] & same[1:-1] & (up[2:] != up[1:-1])
    return int((rec | turn).sum())


def check_counts(info, b_g, prob):
    runs, ivs, recs = layout_counts(b_g.reshape(prob.n), prob.n_bins, info.hist_layout)
    assert (info.hist_intervals, info.hist_records) == (ivs, recs)
    # the record stream may skip building the point stream (runs then read 0)
    assert info.hist_runs == runs or (info.hist_stream == 2 and info.hist_runs == 0)


def run_stream(prob, kind, rows=None):
    from paper_1908_11246_gb300 import vup
    g = vup.Grid(prob.n, prob.lo, prob.hi)
    g.eval_model(prob.model_id, prob.theta, prob.n_bins, prob.n_moments)
    g.set_hist_stream(kind)
    dd = vup.densities_to_device(prob.dens)
    _, _, hs = g.propagate(dd, "fp32", False, False, True)
    g.sync()
    info = g.info()
    b_g = g.array("bins").cpu().numpy()
    hs = hs.cpu().numpy()
    g.close()
    return hs if rows is None else hs[rows], info, b_g


@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
def test_point_and_interval_streams_match_oracle(prob):
    res = O.solve(prob, threads=Hp.oracle_threads())
    amb = Hp.ambiguous_points(res["y"], res["bins"], prob.n_bins)
    amb_mass = 0.0
    if amb.any():
        for k in range(prob.K):
            W, _ = O.weights(prob.n, prob.lo, prob.hi, prob.dens, k)
            amb_mass = max(amb_mass, float(W[amb].sum()))
    out = {}
    for kind in (0, 1, 2):
        hs, info, b_g = run_stream(prob, kind)
        assert info.hist_stream == kind
        Hp.check_hist(hs, res["hist"], amb_mass)
        # the device's run, interval and record counts for its chosen layout, from its own bins
        check_counts(info, b_g, prob)
        out[kind] = hs
    # the orders of summation agree within the sum of their bounds
    for kind in (1, 2):
        assert np.abs(out[0].astype(np.float64) - out[kind]).max() <= 2 * (1e-6 + amb_mass)


@pytest.mark.parametrize("name,expect", [("c2", (1, 2)), ("c3", (0, 0)), ("c4", (1, 2))])
def test_automatic_choice_takes_the_cheaper_stream(name, expect):
    """Full-size workloads.  c2 / c4: gathering axis 0 gives runs of ~9 / ~18
    points in ~1.07 intervals each and ~6 intervals per record, so layout
    1's record stream is cheapest.  c3 (3-D): intervals average 1.8 points and
    records 1.6 intervals, so the point stream is."""
    prob = I.config(name)
    rows = np.array([0, 1, 4097, prob.K - 1])
    hs, info, b_g = run_stream(prob, -1, rows=rows)
    assert (info.hist_layout, info.hist_stream) == expect
    check_counts(info, b_g, prob)
    res = O.solve(prob, rows=rows, threads=Hp.oracle_threads())
    Hp.check_hist(hs, res["hist"])


def test_stream_choice_argument_errors():
    from paper_1908_11246_gb300 import vup
    g = vup.Grid((16,), (0.0,), (1.0,))
    with pytest.raises(vup.VUPError):
        g.set_hist_stream(1)  # 1-D grids have no layout stream
    g.close()
    g = vup.Grid((16, 8), (0.0, 0.0), (1.0, 1.0))
    for bad in (-2, 3):
        with pytest.raises(vup.VUPError):
            g.set_hist_stream(bad)
    g.set_hist_stream(0)  # before a model: kept for the next one
    g.close()
