"""The no-allocation row sort (dm_sort_rows_static) against an independent sort of its input.

dm_sort_rows_static exists for callers that cannot allocate device memory at the moment they
sort (cudaMalloc/cudaFree would synchronise the device under a latency-bound serving thread,
or a host framework's allocator already holds the memory and hands out fixed buffers). Its
temporaries live in one fixed device array inside the library, so these tests check the
result against numpy's stable lexicographic sort of the same input on two calls in a row
through that shared array, at the row limit (which fills every scratch region and takes the
multi-block scan), and that a call allocates no device memory; in a fresh process or after
every other test.

The file name sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_2508_21287_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


def _sort_on_device(B, torch, rows, scores, bits):
    n, w = rows.shape
    rows_in = torch.from_numpy(np.ascontiguousarray(rows)).cuda()
    sc_in = torch.from_numpy(np.ascontiguousarray(scores)).cuda()
    rows_out = torch.full_like(rows_in, -1)
    sc_out = torch.full_like(sc_in, -1.0)
    stream = torch.cuda.current_stream()

    def call():
        B.dm_sort_rows_static(rows_in.data_ptr(), sc_in.data_ptr(), n, w, bits, rows_out.data_ptr(),
                              sc_out.data_ptr(), stream)
    return call, rows_out, sc_out


def _expect(rows, scores):
    order = np.lexsort(rows.T[::-1])  # stable: equal rows keep their input order, as the radix sort
    return rows[order], scores[order]


def test_static_sort_matches_numpy_twice(B):
    torch = pytest.importorskip("torch")
    g = I.heavy_hex(4, 6)
    bits = int(g.n - 1).bit_length()
    for call_no, p in enumerate((I.path(12), I.sub_patch(g, 20, 5))):
        with B.Context(0) as ctx:
            rows, scores, cnt, _ = ctx.plan(ctx.load(I.lognormal_weights(g, seed=3)), p).all()
        rng = np.random.default_rng(call_no)
        perm = rng.permutation(cnt)
        rows_p, sc_p = rows[perm], scores[perm]
        call, rows_out, sc_out = _sort_on_device(B, torch, rows_p, sc_p, bits)
        want_rows, want_sc = _expect(rows_p, sc_p)
        # the embeddings are distinct, so the sorted shuffle is the allocating path's canonical output
        assert np.array_equal(want_rows, rows) and np.array_equal(want_sc, scores)
        for _ in range(2):  # two calls in a row through the shared scratch array
            rows_out.fill_(-1)
            call()
            torch.cuda.synchronize()
            assert np.array_equal(rows_out.cpu().numpy(), want_rows)
            assert np.array_equal(sc_out.cpu().numpy(), want_sc)


@pytest.mark.parametrize("n,w,bits", [(1 << 20, 3, 20), (16385, 2, 14), (70000, 5, 9), (1, 4, 8)])
def test_static_sort_limits_and_no_allocation(B, n, w, bits):
    # n = 2^20 is the largest accepted size; 16385 and 70000 rows take the multi-block scan of
    # the digit histograms; 9-bit ids over 5 columns give many equal rows (stability)
    torch = pytest.importorskip("torch")
    assert B.DM_SORT_STATIC_MAX_ROWS == 1 << 20
    rng = np.random.default_rng(n + w)
    rows = rng.integers(0, 1 << bits, size=(n, w), dtype=np.int32)
    scores = rng.random(n, dtype=np.float32)
    call, rows_out, sc_out = _sort_on_device(B, torch, rows, scores, bits)
    call()  # warm: the library's device code is loaded and the scratch address looked up
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    rows_out.fill_(-1)
    call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0
    want_rows, want_sc = _expect(rows, scores)
    assert np.array_equal(rows_out.cpu().numpy(), want_rows)
    assert np.array_equal(sc_out.cpu().numpy(), want_sc)


def test_static_sort_rejects_oversize(B):
    with pytest.raises(B.DMError) as e:
        B.dm_sort_rows_static(16, None, B.DM_SORT_STATIC_MAX_ROWS + 1, 4, 8, 16, None)
    assert e.value.code == B.DM_E_CAPACITY
    with pytest.raises(B.DMError) as e:
        B.dm_sort_rows_static(16, None, 10, 65, 8, 16, None)
    assert e.value.code == B.DM_E_INVAL
