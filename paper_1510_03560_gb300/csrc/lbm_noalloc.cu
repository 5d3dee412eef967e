// lbm_mass_noalloc: the FP64 per-component mass reduction for callers that
// cannot allocate device memory.  Its scratch (per-block partial sums and
// the two totals) is a fixed-size array that lives in the library image on
// every GPU that loads it, instead of memory obtained from cudaMalloc or a
// caller's allocator.
#include <cstdint>
#include <cstdio>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

// Scratch of lbm_mass_noalloc: LBM_NOALLOC_MAX_BLOCKS x 2 partial sums, then
// the 2 totals.  Every GPU that loads the library holds one copy (1 MiB)
// until the process exits.  Host code must not pass this name to a kernel:
// on the host it is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
constexpr long long kPartials = (long long)LBM_NOALLOC_MAX_BLOCKS * 2;
static __device__ __align__(256) double g_noalloc_scratch[kPartials + 2];

// Errors are reported through lbm_last_error(NULL).
int fail(int code, const char *what, cudaError_t e)
{
    char msg[256];
    snprintf(msg, sizeof msg, "lbm_mass_noalloc: %s%s%s", what, e == cudaSuccess ? "" : ": ",
             e == cudaSuccess ? "" : cudaGetErrorString(e));
    set_global_error(msg);
    return code;
}

// Per-block sums over the non-solid cells, one CTA per block.
__global__ void __launch_bounds__(CELLS) k_noalloc_partial(const float *f, const uint32_t *solid,
                                                           int nblocks, int ncomp, double *partial)
{
    __shared__ double red[CELLS / 32][2];
    const int c = threadIdx.x;
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const bool is_solid =
            solid ? ((solid[(size_t)b * MASK_WORDS + (c >> 5)] >> (c & 31)) & 1u) : false;
        double m[2] = {0.0, 0.0};
        for (int a = 0; a < ncomp; ++a) {
            if (is_solid) continue;
            const float *src = f + ((size_t)b * ncomp + a) * Q * CELLS + c;
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += (double)src[i * CELLS];
            m[a] = acc;
        }
        for (int a = 0; a < 2; ++a)
            for (int o = 16; o > 0; o >>= 1) m[a] += __shfl_down_sync(0xffffffffu, m[a], o);
        if ((c & 31) == 0) {
            red[c >> 5][0] = m[0];
            red[c >> 5][1] = m[1];
        }
        __syncthreads();
        if (c < 2) {
            double t = 0.0;
            for (int w = 0; w < CELLS / 32; ++w) t += red[w][c];
            partial[(size_t)b * 2 + c] = t;
        }
        __syncthreads();
    }
}

// Fixed-order sum of the partials into total[0..1].
__global__ void __launch_bounds__(1024) k_noalloc_total(const double *partial, int nblocks,
                                                        double *total)
{
    __shared__ double red[1024][2];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int i = t; i < nblocks; i += 1024) {
        s0 += partial[(size_t)i * 2];
        s1 += partial[(size_t)i * 2 + 1];
    }
    red[t][0] = s0;
    red[t][1] = s1;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (t < w) {
            red[t][0] += red[t + w][0];
            red[t][1] += red[t + w][1];
        }
        __syncthreads();
    }
    if (t < 2) total[t] = red[0][t];
}

// Device address of the scratch array on the current device, looked up at
// every call with that device current: after a cudaDeviceReset the library's
// module is loaded again and the array may move, so no address is kept from
// one call to the next.
int scratch_for_current_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaGetSymbolAddress", e);
    *out = (double *)p;
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_mass_noalloc(const float *f, const uint32_t *solid, long long nblocks, int ncomp,
                                double *mass, void *stream)
{
    if (!f || !mass) return fail(LBM_EINVAL, "f and mass are required", cudaSuccess);
    if (ncomp != 1 && ncomp != 2) return fail(LBM_EINVAL, "ncomp must be 1 or 2", cudaSuccess);
    if (nblocks < 1 || nblocks > LBM_NOALLOC_MAX_BLOCKS)
        return fail(LBM_EINVAL, "nblocks must be in 1..LBM_NOALLOC_MAX_BLOCKS (65536)", cudaSuccess);
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 1, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaGetDevice", e);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaDeviceGetAttribute", e);
    const int grid = (int)(nblocks < 4LL * sms ? nblocks : 4LL * sms);
    k_noalloc_partial<<<grid, CELLS, 0, s>>>(f, solid, (int)nblocks, ncomp, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "partial-sum launch", e);
    k_noalloc_total<<<1, 1024, 0, s>>>(scratch, (int)nblocks, scratch + kPartials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "total launch", e);
    double out[2] = {0.0, 0.0};
    e = cudaMemcpyAsync(out, scratch + kPartials, sizeof out, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "result copy", e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "stream synchronize", e);
    for (int a = 0; a < ncomp; ++a) mass[a] = out[a];
    return LBM_OK;
}

