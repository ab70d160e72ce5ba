"""The allocation-free Z-sum entry point (qv_zsums_noalloc) must agree with the
handle-based reductions (qv_norm2 / qv_expect_z) it mirrors.

It exists for callers that cannot allocate device memory when they need the
result -- code being recorded into a CUDA graph, latency-critical loops where
cudaMalloc/cudaFree would block or synchronise, or processes whose memory is
handed out by a pool they do not own -- so it keeps its partial sums in one
fixed device array inside the library. This file runs last (pytest collects
it after the others) and passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2508_15545_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc_sums(qv, torch, h):
    n, dt, ptr = qv.qv_info(h)
    out = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    qv.qv_zsums_noalloc(ptr, n, dt, stream, out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("n", [5, 13, 14, 20, 26])
def test_noalloc_matches_handle_reductions_twice(qvlib, cuda, dtype, n):
    qv, torch = qvlib, cuda
    stream = torch.cuda.current_stream()
    h = qv.qv_create(n, dtype, stream)
    tol = 1e-7 if dtype == 0 else 1e-13
    try:
        # two calls in a row on two different states: the second must not see
        # anything the first left in the shared array
        for call, seed in enumerate((11 + n, 23 + n)):
            gates = W.random_circuit(n, 2, seed)
            qv.qv_set_basis(h, 0)
            qv.qv_apply_circuit(h, gates, mode=qv.QV_MODE_PLAIN)
            sums = _noalloc_sums(qv, torch, h)
            assert np.all(np.isfinite(sums)), call
            norm = qv.qv_norm2(h)
            ez, _ = qv.qv_expect_z(h)
            assert sums[0] == pytest.approx(norm, abs=tol)
            assert np.max(np.abs((sums[0] - 2 * sums[1:]) - ez)) <= 2 * tol, call
    finally:
        qv.qv_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_limit(qvlib, cuda):
    qv, torch = qvlib, cuda
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(qv.QvError) as e:
        qv.qv_zsums_noalloc(buf.data_ptr(), 31, qv.QV_C64, torch.cuda.current_stream(), out.data_ptr())
    assert e.value.status == qv.QV_ERR_ARG and "outside [1, 30]" in str(e.value)
    with pytest.raises(qv.QvError):
        qv.qv_zsums_noalloc(0, 4, qv.QV_C64, None, out.data_ptr())


def test_noalloc_after_a_larger_call_reads_only_its_own_partials(qvlib, cuda):
    """A 26-qubit call fills more of the fixed array than a 20-qubit call on
    another state uses next; the smaller call must still give its own sums."""
    qv, torch = qvlib, cuda
    stream = torch.cuda.current_stream()
    big, small = qv.qv_create(26, 0, stream), qv.qv_create(20, 0, stream)
    try:
        qv.qv_apply_circuit(big, W.random_circuit(26, 2, 5), mode=qv.QV_MODE_PLAIN)
        qv.qv_apply_circuit(small, W.random_circuit(20, 2, 6), mode=qv.QV_MODE_PLAIN)
        for h in (big, small):
            sums = _noalloc_sums(qv, torch, h)
            ez, _ = qv.qv_expect_z(h)
            assert sums[0] == pytest.approx(qv.qv_norm2(h), abs=1e-7)
            assert np.max(np.abs((sums[0] - 2 * sums[1:]) - ez)) <= 2e-7
    finally:
        qv.qv_destroy(big)
        qv.qv_destroy(small)


def test_noalloc_at_its_limit_30_qubits(qvlib, cuda):
    """n = 30, the largest size the fixed array holds (all 65,536 blocks of
    partials), complex64, against qv_expect_z on the same state."""
    qv, torch = qvlib, cuda
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << 30) + (2 << 30):
        pytest.skip("needs 10 GiB of free device memory")
    h = qv.qv_create(30, 0, torch.cuda.current_stream())
    try:
        qv.qv_apply_circuit(h, W.random_circuit(30, 1, 9), mode=qv.QV_MODE_FUSED)
        sums = _noalloc_sums(qv, torch, h)
        ez, _ = qv.qv_expect_z(h)
        assert sums[0] == pytest.approx(qv.qv_norm2(h), abs=1e-7)
        assert np.max(np.abs((sums[0] - 2 * sums[1:]) - ez)) <= 2e-7
    finally:
        qv.qv_destroy(h)

