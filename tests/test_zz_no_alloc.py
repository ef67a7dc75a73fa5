"""The no-allocation transform, checked against the plan-based transform.

etd_transform_noalloc is for callers that must not allocate device memory
while they run: a host framework's caching allocator has reserved the GPU's
memory (an extra cudaMalloc could fail or fragment it), or the caller sits in
a latency-critical loop where cudaFree's device-wide synchronisation would
stall other streams. Its workspace is a fixed array inside the library that
every call shares, so this file checks two calls in a row, each against
etd_transform of an FP32 plan on the same input. It runs last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from paper_2601_06849_gb300 import etd, inputs


@pytest.mark.gpu
@pytest.mark.parametrize("d,n,ncomp", [(2, 200, 2), (3, 40, 1), (2, 37, 1), (3, 33, 2)])
def test_noalloc_matches_plan_transform_twice(d, n, ncomp):
    torch = need_gpu()
    stream = torch.cuda.current_stream()
    plan = etd.Plan(d, n, 0.01, 0.0, 1e-3, precision="fp32", reaction="linear", n_comp=ncomp, stream=stream)
    for call in range(2):
        x = torch.tensor(inputs.random_field((ncomp,) + (n,) * d, workload=60, sub=100 * n + call),
                         dtype=torch.float32, device="cuda")
        ref = plan.transform(x)
        out = torch.full_like(x, float("nan"))
        etd.etd_transform_noalloc(d, n, ncomp, x.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert rel_err(out.double().cpu().numpy(), ref.double().cpu().numpy()) < 1e-5
    plan.close()


def test_noalloc_rejects_sizes_beyond_the_static_workspace():
    import __graft_entry__

    __graft_entry__.build()
    for d, n, ncomp in [(2, 4096, 1), (3, 200, 1), (2, 1448, 2)]:
        need = n * n + (2 if d == 3 else 1) * ncomp * n ** d
        assert need > etd.ETD_NOALLOC_MAX_ELEMS
        with pytest.raises(etd.EtdError) as ei:
            etd.etd_transform_noalloc(d, n, ncomp, 256, 256, 0)
        assert ei.value.status == etd.ETD_ERR_INVALID_ARG
        assert "ETD_NOALLOC_MAX_ELEMS" in str(ei.value)
