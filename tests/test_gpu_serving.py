"""The request loop (continuous batching) on the GPU: requests of different
sizes submitted while others run give, each, the same result as the request
run alone through bsm_multiply (bit for bit: the same kernels on the same data)
and the oracle's pattern and values."""
import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


def alone(bsm_lib, A, eps, precision=0):
    with bsm_lib.Context(0) as ctx:
        dA = ctx.from_blocks(A)
        dC = ctx.empty(A.row_sizes, A.col_sizes)
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True, precision=precision)
        r, c = dC.pattern()
        return r, c, dC.values()


def drain(srv, ids, limit=100000):
    for _ in range(limit):
        srv.progress()
        if all(srv.poll(i)[0] >= 2 for i in ids):
            return
    raise AssertionError("requests did not finish")


def test_alone_vs_mix(bsm_lib, oracle_mod):
    eps = 1e-10
    sizes = [8, 40, 16, 64, 24, 8, 32, 12]
    systems = [synth.water(n, seed=1000 + r) for r, n in enumerate(sizes)]
    with bsm_lib.Server(0, slots=3, hbm_budget=2 << 30) as srv:
        ids = [srv.submit(systems[0], eps), srv.submit(systems[1], eps)]
        srv.progress()  # the first two start; the rest arrive while they run
        for A in systems[2:]:
            ids.append(srv.submit(A, eps))
            srv.progress()
        drain(srv, ids)
        info = srv.info()
        assert info["completed"] == len(systems) and info["bytes_peak"] <= 2 << 30
        results = [srv.take(i) for i in ids]
    for A, (r, c, v) in zip(systems, results):
        ra, ca, va = alone(bsm_lib, A, eps)
        assert np.array_equal(r, ra) and np.array_equal(c, ca)
        assert np.array_equal(v, va)  # same kernels, same data: identical
        ref = oracle_mod.multiply(A, A, eps=eps)
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(v, ref.values) <= 1e-12


def test_budget_admission_and_fifo(bsm_lib):
    """A small budget forces requests to wait for memory: never more held than
    the budget, every request completes, and a request larger than the whole
    budget is refused at submission."""
    eps = 1e-10
    systems = [synth.water(24, seed=2000 + r) for r in range(4)]
    # the footprint bound of one such request, as the server accounts it: the
    # peak of a server that ran it alone
    with bsm_lib.Server(0, slots=1, hbm_budget=8 << 30) as srv:
        i0 = srv.submit(systems[0], eps)
        drain(srv, [i0])
        F = srv.info()["bytes_peak"]
        srv.take(i0)
    assert F > 0
    budget = int(2.5 * F)  # room for two requests at a time
    with bsm_lib.Server(0, slots=4, hbm_budget=budget) as srv:
        ids = [srv.submit(A, eps) for A in systems]
        info = srv.info()
        assert info["running"] <= 2  # memory, not lanes, limits
        drain(srv, ids)
        info = srv.info()
        assert info["bytes_peak"] <= budget and info["completed"] == 4
        with pytest.raises(bsm_lib.BsmError) as e:
            srv.submit(synth.water(96, seed=1), eps)
        assert e.value.name == "NOMEM"
        for i in ids:
            srv.take(i)
        assert srv.info()["bytes_in_use"] == 0


def test_result_views_and_release(bsm_lib, oracle_mod):
    """bsm_server_result hands out the result in place (page-locked host memory)
    and bsm_server_release returns it; the views equal a lone multiply's result."""
    eps = 1e-10
    systems = [synth.water(n, seed=3000 + n) for n in (12, 30, 20)]
    with bsm_lib.Server(0, slots=2, hbm_budget=2 << 30) as srv:
        ids = [srv.submit(A, eps) for A in systems]
        drain(srv, ids)
        for A, i in zip(systems, ids):
            r, c, v = srv.result(i)
            ra, ca, va = alone(bsm_lib, A, eps)
            assert np.array_equal(r, ra) and np.array_equal(c, ca) and np.array_equal(v, va)
            srv.release(i)
            with pytest.raises(bsm_lib.BsmError):
                srv.result(i)
        assert srv.info()["bytes_in_use"] == 0


def test_submit_from_several_threads(bsm_lib):
    """Requests submitted from three threads at once while the main thread
    polls: all complete, each with the result of the request run alone."""
    import threading

    eps = 1e-10
    systems = [synth.water(n, seed=4000 + n) for n in (6, 10, 14, 18, 22, 26)]
    ids = [None] * len(systems)
    with bsm_lib.Server(0, slots=2, hbm_budget=2 << 30) as srv:
        def client(lo):
            for j in range(lo, len(systems), 3):
                ids[j] = srv.submit(systems[j], eps)

        threads = [threading.Thread(target=client, args=(t,)) for t in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert len(set(ids)) == len(systems)
        drain(srv, ids)
        for A, i in zip(systems, ids):
            r, c, v = srv.take(i)
            ra, ca, va = alone(bsm_lib, A, eps)
            assert np.array_equal(r, ra) and np.array_equal(c, ca) and np.array_equal(v, va)
        assert srv.info()["bytes_in_use"] == 0


@pytest.mark.parametrize("prec", [1, 2])
def test_split_precision_server(bsm_lib, oracle_mod, prec):
    """A server in a split precision (BF16x3, TF32x2): every result equals the
    same multiply run alone in that precision (same kernels: bit for bit) and
    the oracle within the split bound on water."""
    eps = 1e-10
    systems = [synth.water(n, seed=5000 + n) for n in (10, 36, 18, 27)]
    with bsm_lib.Server(0, slots=2, precision=prec, hbm_budget=2 << 30) as srv:
        ids = [srv.submit(A, eps) for A in systems]
        drain(srv, ids)
        for A, i in zip(systems, ids):
            r, c, v = srv.take(i)
            ra, ca, va = alone(bsm_lib, A, eps, precision=prec)
            assert np.array_equal(r, ra) and np.array_equal(c, ca) and np.array_equal(v, va)
            ref = oracle_mod.multiply(A, A, eps=eps)
            assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
            assert H.rel_frobenius(v, ref.values) <= 1e-5


def _permuted(A, rng):
    """The same matrix with its block list in random order (values moved with
    their blocks)."""
    lens = A.row_sizes.astype(np.int64)[A.blk_row] * A.col_sizes.astype(np.int64)[A.blk_col]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    p = rng.permutation(len(lens))
    vals = np.concatenate([A.values[off[b]:off[b + 1]] for b in p]) if len(p) else A.values
    return synth.BlockMatrix(A.row_sizes, A.col_sizes, A.blk_row[p], A.blk_col[p], vals)


def test_small_requests_share_multiplies(bsm_lib, oracle_mod):
    """Small requests queued together run as one multiply of their
    block-diagonal matrix: fewer multiplies than requests, and each request's
    part equals the request multiplied alone, bit for bit."""
    eps = 1e-10
    sizes = [8, 12, 6, 16, 10, 8, 14, 4, 9, 11]
    systems = [synth.water(n, seed=6000 + r) for r, n in enumerate(sizes)]
    B = synth.water(128, seed=6100)
    with bsm_lib.Server(0, slots=1, hbm_budget=4 << 30) as srv:
        # a larger request first holds the only lane while the small ones queue
        big = srv.submit(B, eps)
        while srv.poll(big)[0] == 0:
            pass
        ids = [srv.submit(A, eps) for A in systems]
        drain(srv, [big] + ids)
        info = srv.info()
        assert info["completed"] == len(systems) + 1
        assert info["batches"] < len(systems) + 1  # some of them shared a multiply
        srv.release(big)
        results = [srv.take(i) for i in ids]
    for A, (r, c, v) in zip(systems, results):
        ra, ca, va = alone(bsm_lib, A, eps)
        assert np.array_equal(r, ra) and np.array_equal(c, ca)
        assert np.array_equal(v, va)
        ref = oracle_mod.multiply(A, A, eps=eps)
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(v, ref.values) <= 1e-12


def test_unsorted_submission_and_duplicates(bsm_lib, oracle_mod):
    """A block list in any order gives the result of the sorted one; a block
    listed twice is refused at submission."""
    eps = 1e-10
    rng = np.random.default_rng(5)
    A = synth.water(20, seed=6200)
    P = _permuted(A, rng)
    with bsm_lib.Server(0, slots=2, hbm_budget=2 << 30) as srv:
        ids = [srv.submit(P, eps), srv.submit(A, eps)]
        drain(srv, ids)
        r1, c1, v1 = srv.take(ids[0])
        r2, c2, v2 = srv.take(ids[1])
        assert np.array_equal(r1, r2) and np.array_equal(c1, c2) and np.array_equal(v1, v2)
        ref = oracle_mod.multiply(A, A, eps=eps)
        assert np.array_equal(r1, ref.blk_row) and H.rel_frobenius(v1, ref.values) <= 1e-12
        n0 = int(A.row_sizes[A.blk_row[0]]) * int(A.col_sizes[A.blk_col[0]])
        D = synth.BlockMatrix(A.row_sizes, A.col_sizes, np.append(A.blk_row, A.blk_row[0]),
                              np.append(A.blk_col, A.blk_col[0]), np.append(A.values, A.values[:n0]))
        with pytest.raises(bsm_lib.BsmError) as e:
            srv.submit(D, eps)
        assert e.value.name == "DUPLICATE_BLOCK"
        assert srv.info()["bytes_in_use"] == 0


def test_small_request_passes_earlier_large_one(bsm_lib):
    """Earliest deadline first: with one lane busy, a small request submitted
    just after a large one is admitted before it."""
    eps = 1e-10
    S = [synth.water(1024, seed=6300), synth.water(256, seed=6301), synth.water(8, seed=6302)]
    with bsm_lib.Server(0, slots=1, hbm_budget=48 << 30) as srv:
        # a request of the large one's size first: its page-locked block is then
        # cached, so that submitting the large one below takes a copy, no allocation
        w = srv.submit(S[1], eps)
        drain(srv, [w])
        srv.release(w)
        first = srv.submit(S[0], eps)
        while srv.poll(first)[0] == 0:  # until it holds the only lane
            pass
        large = srv.submit(S[1], eps)
        small = srv.submit(S[2], eps)
        assert srv.poll(first)[0] == 1  # both queued while the lane is busy
        order = []
        for _ in range(10 ** 7):
            srv.progress()
            for i in (first, large, small):
                if i not in order and srv.poll(i)[0] >= 2:
                    order.append(i)
            if len(order) == 3:
                break
        assert order == [first, small, large]
        for i in order:
            srv.release(i)


def test_large_sliced_request_beside_small_ones(bsm_lib):
    """A large request (numeric phase in slices, the next slice held back while
    small batches run) and small requests submitted while it runs: every result
    is bit for bit the request run alone, and each request's time splits into
    submit, queue and run parts that add up to its latency."""
    eps = 1e-10
    large = synth.water(1024, seed=6400)
    small = [synth.water(n, seed=6401 + r) for r, n in enumerate([8, 24, 16, 32, 12, 40])]
    with bsm_lib.Server(0, slots=3, hbm_budget=48 << 30) as srv:
        first = srv.submit(large, eps)
        while srv.poll(first)[0] == 0:
            pass
        ids = []
        for A in small:
            ids.append(srv.submit(A, eps))
            srv.progress()
        pending = [i for i in ids if srv.poll(i)[0] < 2]
        if pending:  # not finished yet: no timing
            with pytest.raises(bsm_lib.BsmError):
                srv.timing(pending[0])
        drain(srv, [first] + ids)
        with pytest.raises(bsm_lib.BsmError):
            srv.timing(10 ** 9)
        for i in [first] + ids:
            state, lat, _, _ = srv.poll(i)
            assert state == 2
            t_sub, t_wait, t_run = srv.timing(i)
            assert min(t_sub, t_wait, t_run) >= 0.0 and t_run > 0.0
            assert abs(t_sub + t_wait + t_run - lat) <= 1e-6 * max(lat, 1.0)
        results = [srv.take(i) for i in [first] + ids]
    for A, (r, c, v) in zip([large] + small, results):
        ra, ca, va = alone(bsm_lib, A, eps)
        assert np.array_equal(r, ra) and np.array_equal(c, ca)
        assert np.array_equal(v, va)


def test_borrowed_submission(bsm_lib, oracle_mod):
    """bsm_server_submit_borrowed: the values are read from the caller's array
    when the request runs (no copy at submission). Each result equals the
    request run alone, also beside copied submissions and in merged batches;
    an unsorted block list is refused."""
    eps = 1e-10
    systems = [synth.water(n, seed=6500 + r) for r, n in enumerate([24, 8, 40, 16, 1024])]
    with bsm_lib.Server(0, slots=3, hbm_budget=48 << 30) as srv:
        ids = [srv.submit(A, eps, borrow=(r % 2 == 0)) for r, A in enumerate(systems)]
        drain(srv, ids)
        results = [srv.take(i) for i in ids]
        assert not srv._borrowed  # taken requests hold no borrowed arrays
        P = _permuted(systems[0], np.random.default_rng(9))
        with pytest.raises(bsm_lib.BsmError) as e:
            srv.submit(P, eps, borrow=True)
        assert e.value.name == "INVALID_ARG"
    for A, (r, c, v) in zip(systems, results):
        ra, ca, va = alone(bsm_lib, A, eps)
        assert np.array_equal(r, ra) and np.array_equal(c, ca)
        assert np.array_equal(v, va)
    ref = oracle_mod.multiply(systems[0], systems[0], eps=eps)
    assert np.array_equal(results[0][0], ref.blk_row) and H.rel_frobenius(results[0][2], ref.values) <= 1e-12
