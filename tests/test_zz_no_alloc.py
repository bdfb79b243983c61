"""The no-allocation row sort (dm_sort_rows_static) against the library's own canonical output.

dm_sort_rows_static exists for callers that cannot allocate device memory at the moment they
sort (cudaMalloc/cudaFree would synchronise the device under a latency-bound serving thread,
or a host framework's allocator already holds the memory and hands out fixed buffers). Its
temporaries live in one fixed device array inside the library, so this test checks that the
result is right on two calls in a row through that shared array, in a fresh process or after
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


def _canonical(B, ctx, gid, p):
    rows, scores, cnt, _ = ctx.plan(gid, p).all()
    assert rows.shape == (cnt, p.n)
    return rows, scores


def test_static_sort_matches_match_output_twice(B):
    torch = pytest.importorskip("torch")
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=3)
    bits = int(g.n - 1).bit_length()
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        for call, p in enumerate((I.path(12), I.sub_patch(g, 20, 5))):
            want_rows, want_scores = _canonical(B, ctx, gid, p)
            perm = np.random.default_rng(call).permutation(len(want_rows))
            rows_in = torch.from_numpy(np.ascontiguousarray(want_rows[perm])).cuda()
            sc_in = torch.from_numpy(np.ascontiguousarray(want_scores[perm])).cuda()
            rows_out = torch.full_like(rows_in, -1)
            sc_out = torch.full_like(sc_in, -1.0)
            stream = torch.cuda.current_stream()
            B.dm_sort_rows_static(rows_in.data_ptr(), sc_in.data_ptr(), len(want_rows), p.n, bits,
                                  rows_out.data_ptr(), sc_out.data_ptr(), stream)
            torch.cuda.synchronize()
            got_rows = rows_out.cpu().numpy()
            got_scores = sc_out.cpu().numpy()
            assert np.array_equal(got_rows, want_rows)
            np.testing.assert_allclose(got_scores, want_scores, rtol=1e-5, atol=0)


def test_static_sort_rejects_oversize(B):
    with pytest.raises(B.DMError) as e:
        B.dm_sort_rows_static(16, None, B.DM_SORT_STATIC_MAX_ROWS + 1, 4, 8, 16, None)
    assert e.value.code == B.DM_E_CAPACITY
    with pytest.raises(B.DMError) as e:
        B.dm_sort_rows_static(16, None, 10, 65, 8, 16, None)
    assert e.value.code == B.DM_E_INVAL
