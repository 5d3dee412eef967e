// The FP32 storage form of the step kernels (lbm_step.cuh), the dispatch
// of the launch wrappers of lbm_internal.h on the storage form, and the
// final FP64 mass reduction shared by every form.
#include "lbm_step.cuh"

namespace lbm {
namespace {

// Fixed-order sum of the per-slot partial masses into out[0..1], taken in
// block order, so that the result does not depend on the slot numbering.
__global__ void __launch_bounds__(1024) k_mass_final(KParams kp, const double *partial, int n, double *out)
{
    __shared__ double red[1024][2];
    const int t = threadIdx.x;
    const int nb = kp.nbx * kp.nby * kp.nbz;
    double s0 = 0.0, s1 = 0.0;
    for (int b = t; b < nb; b += 1024) {
        const int i = kp.slot_of[b];
        if (i < 0 || i >= n) continue;
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
    if (t < 2) out[t] = red[0][t];
}

// Frontier blocks (unmeshed, not all solid, with a meshed face or edge
// neighbour) of the first *nsnap slots, each listed once: one warp per
// slot, one lane per neighbour.
__global__ void __launch_bounds__(256) k_frontier(KParams kp, const int *nsnap, unsigned *mark, int *list,
                                                  int *count)
{
    const int n = *nsnap;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    const bool face_or_edge = lane < 27 && lane != 13 && (dx * dx + dy * dy + dz * dz) <= 2;
    for (int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); slot < n; slot += nwarps) {
        if (!face_or_edge) continue;
        if (kp.nbr[(size_t)slot * NBR_STRIDE + lane] != AMBIENT) continue;
        const int nid = neighbour_of(kp, kp.block_of[slot], lane);
        if (nid >= 0 && atomicCAS(&mark[nid], 0u, 1u) == 0u) list[atomicAdd(count, 1)] = nid;
    }
}

// Prepare the listed blocks whose probability exceeds thr: their cells'
// solid words (as block creation computes them) into nbits_pre, then the
// flag.  One CTA per block.
__global__ void __launch_bounds__(CELLS) k_prepare(KParams kp, const int *list, const int *count,
                                                   const float *prob, float thr, unsigned *prep,
                                                   uint32_t *nbits_pre)
{
    __shared__ unsigned done;
    const int n = *count;
    const int c = threadIdx.x;
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        const int gid = list[b];
        if (!(prob[b] > thr)) continue;  // the same for the whole CTA
        if (c == 0) done = *(volatile unsigned *)&prep[gid];
        __syncthreads();
        const bool skip = done != 0u;
        __syncthreads();
        if (skip) continue;
        nbits_pre[(size_t)gid * CELLS + c] = cell_bits(kp, gid, c);
        __syncthreads();
        if (c == 0) {
            __threadfence();
            *(volatile unsigned *)&prep[gid] = 1u;
            atomicAdd(&kp.ctrl->prepared, 1ull);
        }
    }
}

// One grid barrier expecting `missing` more CTAs than launched (it can only
// complete when missing is 0), for tests of the bounded wait.
__global__ void __launch_bounds__(128) k_barrier_selftest(Ctrl *ctrl, int missing, long long spins)
{
    grid_sync(ctrl, gridDim.x + (unsigned)missing, spins);
}

const StorageOps &ops_of(const KParams &kp)
{
    switch (kp.storage) {
    case LBM_STORAGE_FP16: return *storage_ops_fp16();
    case LBM_STORAGE_BF16: return *storage_ops_bf16();
    default:
        switch (kp.shape) {
        case 1: return *storage_ops_fp32_16x8x4();
        case 2: return *storage_ops_fp32_16x4x8();
        case 3: return *storage_ops_fp32_32x4x4();
        default: return *storage_ops_fp32();
        }
    }
}

}  // namespace

const StorageOps *storage_ops_fp32() { return Launch<LBM_STORAGE_FP32>::ops(); }

cudaError_t launch_init(const KParams &kp, const float *in_block, int slot0, int nslots, int grid,
                        cudaStream_t s)
{
    return ops_of(kp).init(kp, in_block, slot0, nslots, grid, s);
}

cudaError_t launch_init_finish(const KParams &kp, int nslots, int sms, cudaStream_t s)
{
    return ops_of(kp).init_finish(kp, nslots, sms, s);
}

cudaError_t launch_ambient_slot(const KParams &kp, cudaStream_t s) { return ops_of(kp).ambient_slot(kp, s); }

cudaError_t launch_macro(const KParams &kp, int step, int criterion, int sms, cudaStream_t s)
{
    return ops_of(kp).macro(kp, step, criterion, sms, s);
}

cudaError_t launch_activate(const KParams &kp, int step, int sms, cudaStream_t s)
{
    return ops_of(kp).activate(kp, step, sms, s);
}

cudaError_t launch_collide(const KParams &kp, int step, int sms, cudaStream_t s)
{
    return ops_of(kp).collide(kp, step, sms, s);
}

cudaError_t launch_fused(const KParams &kp, int sms, cudaStream_t s) { return ops_of(kp).fused(kp, sms, s); }

cudaError_t launch_output(const KParams &kp, int rd, int comp, int slot0, int nslots, float *out,
                          int sms, cudaStream_t s)
{
    return ops_of(kp).output(kp, rd, comp, slot0, nslots, out, sms, s);
}

cudaError_t launch_mass(const KParams &kp, int rd, int n, double *partial, double *out, int grid,
                        cudaStream_t s)
{
    cudaError_t e = ops_of(kp).mass_partial(kp, rd, n, partial, grid, s);
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, 1024, 0, s>>>(kp, partial, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sort(const KParams &kp, int sms, cudaStream_t s) { return ops_of(kp).sort(kp, sms, s); }

cudaError_t launch_block_pops(const KParams &kp, int rd, int slot, float *out, cudaStream_t s)
{
    return ops_of(kp).block_pops(kp, rd, slot, out, s);
}

cudaError_t launch_frontier(const KParams &kp, const int *nsnap, unsigned *mark, int *list, int *count,
                            int sms, cudaStream_t s)
{
    k_frontier<<<sms * 4, 256, 0, s>>>(kp, nsnap, mark, list, count);
    return cudaGetLastError();
}

cudaError_t launch_features(const KParams &kp, int par, const int *nsnap, const int *list,
                            const int *count, float *feat, int sms, cudaStream_t s)
{
    return ops_of(kp).features(kp, par, nsnap, list, count, feat, sms, s);
}

cudaError_t launch_prepare(const KParams &kp, const int *list, const int *count, const float *prob,
                           float thr, unsigned *prep, uint32_t *nbits_pre, int sms, cudaStream_t s)
{
    k_prepare<<<sms * 2, CELLS, 0, s>>>(kp, list, count, prob, thr, prep, nbits_pre);
    return cudaGetLastError();
}

cudaError_t launch_run(const KParams &kp, int nsteps, int progressive, int sms, cudaStream_t s)
{
    return ops_of(kp).run(kp, nsteps, progressive, sms, s);
}

int barrier_selftest(int missing, long long spins, int sms)
{
    Ctrl *ctrl = nullptr;
    if (cudaMalloc(&ctrl, sizeof(Ctrl)) != cudaSuccess) return LBM_ENOMEM;
    cudaMemset(ctrl, 0, sizeof(Ctrl));
    void *args[] = {&ctrl, &missing, &spins};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, sms, 128, args, 0, 0);
    int status = LBM_ECUDA;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        Ctrl h{};
        if (cudaMemcpy(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost) == cudaSuccess) status = h.status;
    } else {
        cudaGetLastError();
    }
    cudaFree(ctrl);
    return status;
}

int max_ctas_per_sm_stream_kernels(int storage)
{
    KParams kp{};
    kp.storage = storage;
    return ops_of(kp).ctas_per_sm();
}

}  // namespace lbm
