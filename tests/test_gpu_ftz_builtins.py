"""The pair step takes 1/sqrt(s^2) and the literal reading's quotient from
the flush-to-zero PTX forms `rsqrt.approx.ftz.f32` and `div.approx.ftz.f32`,
on operands that are normal by construction.  This checks, on the GPU, over
every positive normal float, that the rsqrt form equals CUDA's rsqrtf bit for
bit, and that the divide form equals __fdividef wherever the quotient is
normal (they may differ only where it would be subnormal, which max(1, .)
absorbs).  The check kernel is compiled here with NVRTC; it is not part of
the library.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

SRC = r"""
extern "C" __global__ void check(unsigned long long n, unsigned* out) {
    unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long st = (unsigned long long)gridDim.x * blockDim.x;
    for (; i < n; i += st) {
        const float x = __uint_as_float(0x00800000u + (unsigned)i);  // positive normals
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        if (__float_as_uint(r) != __float_as_uint(rsqrtf(x))) atomicAdd(out, 1u);
        // divisors in [0.25, 4), numerators every normal of either sign
        const float y = 0.25f + (float)(i % 1000003ull) * (3.75f / 1000003.f);
        const float xs = (i & 1) ? -x : x;
        float q;
        asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(q) : "f"(xs), "f"(y));
        const float qr = __fdividef(xs, y);
        if (__float_as_uint(q) != __float_as_uint(qr) && !(q == 0.f && qr == 0.f)) {
            atomicAdd(out + 1, 1u);
            if (fabsf(qr) >= 1.17549435e-38f) atomicAdd(out + 2, 1u);
        }
    }
}
"""


def _cubin():
    from cuda.bindings import nvrtc
    err, prog = nvrtc.nvrtcCreateProgram(SRC.encode(), b"ftz_check.cu", 0, [], [])
    assert err == nvrtc.nvrtcResult.NVRTC_SUCCESS
    opts = [b"--gpu-architecture=sm_103a"]
    (err,) = nvrtc.nvrtcCompileProgram(prog, len(opts), opts)
    if err != nvrtc.nvrtcResult.NVRTC_SUCCESS:
        _, n = nvrtc.nvrtcGetProgramLogSize(prog)
        log = b" " * n
        nvrtc.nvrtcGetProgramLog(prog, log)
        raise AssertionError(log.decode(errors="replace"))
    err, n = nvrtc.nvrtcGetCUBINSize(prog)
    assert err == nvrtc.nvrtcResult.NVRTC_SUCCESS
    cubin = b" " * n
    (err,) = nvrtc.nvrtcGetCUBIN(prog, cubin)
    assert err == nvrtc.nvrtcResult.NVRTC_SUCCESS
    nvrtc.nvrtcDestroyProgram(prog)
    return cubin


def test_ftz_forms_match_cuda_functions_on_normal_operands():
    import torch
    from cuda.bindings import driver
    torch.cuda.set_device(0)
    out = torch.zeros(3, dtype=torch.int32, device="cuda")  # also makes torch's context current
    (err,) = driver.cuInit(0)
    assert err == driver.CUresult.CUDA_SUCCESS
    err, mod = driver.cuModuleLoadData(_cubin())
    assert err == driver.CUresult.CUDA_SUCCESS
    err, fn = driver.cuModuleGetFunction(mod, b"check")
    assert err == driver.CUresult.CUDA_SUCCESS
    n = 0x7F7FFFFF - 0x00800000 + 1  # every positive normal float
    args = ((n, out.data_ptr()), (ctypes.c_ulonglong, ctypes.c_void_p))
    (err,) = driver.cuLaunchKernel(fn, 148 * 8, 1, 1, 256, 1, 1, 0, 0, args, 0)
    assert err == driver.CUresult.CUDA_SUCCESS
    torch.cuda.synchronize()
    driver.cuModuleUnload(mod)
    rs_bad, dv_bad, dv_bad_normal = (int(v) for v in out.cpu())
    assert rs_bad == 0
    assert dv_bad_normal == 0
    assert dv_bad < n // 100  # only the subnormal-quotient corner
