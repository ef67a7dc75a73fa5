"""The no-allocation transform, checked against the definition of the transform.

etd_transform_noalloc is for callers that must not allocate device memory
while they run: a host framework's caching allocator has reserved the GPU's
memory (an extra cudaMalloc could fail or fragment it), or the caller sits in
a latency-critical loop where cudaFree's device-wide synchronisation would
stall other streams. Its workspace is a fixed array inside the library that
every call shares, so this file checks two calls in a row, each against the
FP64 definition T(X) = P^T X P (2D) / the three mode products (3D), and that a
call leaves the device's free memory unchanged. It runs last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err, sine_basis
from paper_2601_06849_gb300 import etd, inputs


def reference(x, d):
    P = sine_basis(x.shape[-1])
    if d == 2:
        return np.einsum("yl,cyx,xk->clk", P, x, P, optimize=True)
    return np.einsum("zp,yl,czyx,xk->cplk", P, P, x, P, optimize=True)


def fp32_bound(n, d):
    """Each of the d passes sums n FP32 products (FMA chain, round to nearest);
    with terms of random sign the rounding error of such a sum stays within a
    few sqrt(n) units of 2^-24 relative to the result's scale: 4 sqrt(n) 2^-24
    per pass, d passes (the bound the FP32 path of the step is held to)."""
    return d * 4 * np.sqrt(n) * 2.0 ** -24


@pytest.mark.gpu
@pytest.mark.parametrize("d,n,ncomp", [(2, 200, 2), (3, 40, 1), (2, 37, 1), (3, 33, 2)])
def test_noalloc_matches_definition_twice_without_allocating(d, n, ncomp):
    torch = need_gpu()
    stream = torch.cuda.current_stream()
    xs = [torch.tensor(inputs.random_field((ncomp,) + (n,) * d, workload=60, sub=100 * n + call),
                       dtype=torch.float32, device="cuda") for call in range(2)]
    outs = [torch.full_like(x, float("nan")) for x in xs]
    # the first call on this device looks up the workspace's address (and loads
    # the library's device code if nothing did yet): not measured
    etd.etd_transform_noalloc(d, n, ncomp, xs[0].data_ptr(), outs[0].data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    for call in range(2):
        free0, _ = torch.cuda.mem_get_info()
        etd.etd_transform_noalloc(d, n, ncomp, xs[call].data_ptr(), outs[call].data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, "the call changed the device's free memory"
        ref = reference(xs[call].double().cpu().numpy(), d)
        assert rel_err(outs[call].double().cpu().numpy(), ref) < fp32_bound(n, d)


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
