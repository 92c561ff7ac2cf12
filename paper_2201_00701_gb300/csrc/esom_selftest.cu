// Self-test kernel of the FP64 reciprocal used by the 2x2 solve (drcp: an
// SFU seed refined by two Newton steps), beside CUDA's own division, so a
// test can compare the two over the range of determinants the solve sees.
#include "esom_fused.cuh"

namespace esom {

__global__ void drcp_selftest_kernel(const double *__restrict__ x, long long n,
                                     double *__restrict__ rcp, double *__restrict__ div) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    rcp[i] = drcp(v);
    div[i] = 1.0 / v;
}

cudaError_t launch_drcp_selftest(const double *x, long long n, double *rcp, double *div,
                                 cudaStream_t stream) {
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    drcp_selftest_kernel<<<(unsigned)blocks, 256, 0, stream>>>(x, n, rcp, div);
    return cudaGetLastError();
}

}  // namespace esom
