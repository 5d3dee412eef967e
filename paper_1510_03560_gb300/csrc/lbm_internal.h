// Internal types shared by the host runtime (lbm_capi.cpp) and the kernels
// (lbm_kernels.cu).  Not part of the public C ABI (include/lbm.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace lbm {

constexpr int EDGE = 8;     // cells per block edge of the default 8^3 shape

// Block shapes the step kernels are compiled for (cells along x, y, z; 512
// cells each, x-rows of whole 32-byte sectors).  Index 0 is the default.
struct BlockShape {
    int x, y, z;
};
constexpr int NSHAPES = 4;
constexpr BlockShape BLOCK_SHAPES[NSHAPES] = {{8, 8, 8}, {16, 8, 4}, {16, 4, 8}, {32, 4, 4}};
constexpr int CELLS = 512;  // cells per block
constexpr int Q = 19;       // D3Q19
constexpr int MASK_WORDS = CELLS / 32;
constexpr int HELD_BIT = 19;  // bit of a cell's neighbour word marking a held cell
constexpr int NBR_STRIDE = 32; // ints per row of the neighbour-slot table (27 used)

// slot_of[] values besides a slot index
constexpr int AMBIENT = -1;  // unmeshed block (at least one non-solid cell)
constexpr int SOLIDBLK = -2; // every cell solid, or outside a non-periodic axis

// Device-resident control words.  Counts are double-buffered by step
// parity so that no kernel has to reset a word another kernel of the same
// step still reads.
struct Ctrl {
    int n_active[2];   // meshed blocks at the start of a step of this parity
    int ncand[2];      // candidate blocks found by the criterion
    int status;        // 0, or an LBM_E* code raised on the device
    int fail_step;     // step at which status was raised
    unsigned long long cell_updates;   // 512 x meshed blocks, summed over steps
    unsigned long long fluid_updates;  // fluid cells of meshed blocks, summed over steps
    unsigned long long fluid_active;   // fluid cells of the meshed blocks now
    unsigned long long created;        // blocks created by the criterion
    unsigned long long prepared;       // blocks prepared by the activation proposer
    unsigned long long prepared_hits;  // created blocks that had been prepared
    int step;          // completed steps, advanced on the device by each step
    unsigned collide_done;     // CTAs of the current collide launch that finished
    unsigned bar_count, bar_gen;   // grid barrier of the multi-step kernel
    float psi_amb;     // psi of the ambient density, evaluated on the device
    int check_site;    // checked builds: first failed index check (site id)
    long long check_value;  // and the offending value
    unsigned long long sorted_created;  // `created` at the last renumbering of the slots
    unsigned long long sorts;           // renumberings of the slots in block order
    unsigned macro_done;  // CTAs of the current pass-1 launch that finished
    int sort_go;       // the renumbering under way moves the slots
    int n_sorted;      // A-A: the first n_sorted work items visit kp.order
    // fused step launch (collision of step t + pass 1 of step t + 1)
    int fz_dist;       // neighbour slot distance that covers most slots (the lag)
    unsigned fz_hist_ctas;  // CTAs of k_sort_tables done with the distance histogram
    unsigned long long fz_deferred;  // pass-1 items skipped and redone at the end of their CTA's
                                     // sequence, summed over launches
    unsigned long long fz_waited;    // pass-1 warp items that found a collision unfinished
};

// Neighbour-distance histogram of the fused step's lag: bins of FZ_BIN
// slots, the last one open-ended.  The lag covers the distance of
// FZ_COVER_PERMIL / 1000 of the slots; the others are deferred.
constexpr int FZ_BINS = 1024;
constexpr int FZ_BIN = 8;
constexpr int FZ_COVER_PERMIL = 900;
// Default cap of the lag, in half-block work items: the populations written
// and read during the lag must stay in the 126 MB of L2.
constexpr int FZ_MAX_LAG = 1536;

// Everything a kernel needs, passed by value.
struct KParams {
    int nbx, nby, nbz;
    int per[3];
    int ncomp;
    int capacity;
    int amb_slot;       // == capacity: a slot holding the resting ambient state
                        // (populations in both buffers, first-pass values)
    int progressive;
    int storage;        // LBM_STORAGE_*
    // physics, FP32
    float omega;        // 1 / tau
    float beta, g_self, g_cross;
    float g_ads[2];
    float grav[3];
    float rho_ref[2];
    float S2;           // S^2
    float pr_b, pr_RT, pr_atheta;
    float psi_scale;    // 2 / (c_s^2 g_self), 0 when g_self == 0
    float rho_amb[2];
    float psi_amb;
    float famb[2][Q];   // ambient resting populations w_i rho_amb
    // device memory
    float *f;           // FP32 form: [2][capacity + 1][ncomp][Q][CELLS]
                        // (one buffer with A-A streaming)
    uint32_t *h;        // 16-bit forms: [2][capacity + 1][Q][CELLS] words of
                        // two 16-bit deviations from w_i rho of the reading
                        // cell (component 0 low, component 1 high)
    float4 *mac;        // [capacity + 1][CELLS]: rho0, rho1, psi0, 0 of the
                        // current step; the 16-bit forms keep two of them,
                        // by step parity (mac_stride apart), because the
                        // previous step's densities are the references
    size_t mac_stride;  // 0 (FP32 form) or (capacity + 1) * CELLS
    uint32_t *nbits;    // [capacity][CELLS]: bit i set when cell x - e_i is solid
                        // (bit 0: the cell itself), bit HELD_BIT: held cell
    float *uprev;       // [capacity][ncomp][3][CELLS]; in the 16-bit forms
                        // also the velocity of held cells
    int *slot_of;       // [nblocks]
    int *nbr;           // [capacity][NBR_STRIDE]: slots of the 27 blocks around a slot
    int *block_of;      // [capacity]
    const uint32_t *solid;  // [nblocks][MASK_WORDS]
    const uint32_t *held;   // [nblocks][MASK_WORDS]
    int *cand_list;     // [nblocks]
    unsigned *cand_mark;    // [nblocks]
    int *act_step;      // [nblocks]: step + 1 of creation, 0 initial, -1 unmeshed
    const unsigned *prep;       // [nblocks] or NULL: 1 once nbits_pre holds the block's words
    const uint32_t *nbits_pre;  // [nblocks][CELLS]: solid words prepared by the proposer
    Ctrl *ctrl;
    size_t buf_stride;  // elements (floats or words) per population buffer;
                        // 0 with A-A streaming
    int slot_floats;    // elements per slot: ncomp * Q * CELLS (FP32) or
                        // Q * CELLS (16-bit forms)
    long long barrier_spins;  // bounded wait of a grid barrier or a bulk copy (polls)
    int staged;         // FP32, two components: TMA-staged pass kernels
    int shape;          // index into BLOCK_SHAPES (the FP32 form has all;
                        // the 16-bit forms only 8^3)
    // A-A streaming (FP32, two components): one population array (f, with
    // buf_stride 0, so that both parities address it), updated in place
    int aa;
    float *held_f;          // [held blocks][2][Q][CELLS]: the constant
                            // populations of held cells (A-A only)
    const int *held_rank;   // [nblocks]: row of held_f, -1 without held cells
    int *order;             // A-A: [capacity] slots in block order (the first
                            // ctrl->n_sorted of them); the passes visit them
                            // in this order instead of moving the blocks
    // fused step (FP32, two components, A-B)
    int *cflag;             // [2][capacity * 2]: per step parity and half block, the
                            // warps that have finished its collision
    int *fz_hist;           // [FZ_BINS]: neighbour distances of the slots (renumbering)
    int fz_max_lag;         // cap of the lag in work items
    int strip;              // slot order: strips of this many block rows along y
                            // (each strip in z, y, x order); 0 = block order
    // density partials (FP32, two components, A-B): written by the collision
    // of a step, summed by pass 1 of the next one instead of its pull
    float2 *part;           // [capacity][CELLS]: per cell, the sum of the values it
                            // will pull from its own half block
    float2 *recv;           // [capacity][2][recv_entries]: per half block, what its
                            // neighbour half blocks send to its boundary cells
    int part_in;            // pass 1 sums the partials (where no neighbour block is unmeshed)
    int part_out;           // the collision writes them
};

// Entries of the density partials of one half block (blocks split in two
// along z): one per cell just outside one of its 6 faces or 12 edges (the
// corners are out of reach of D3Q19).
__host__ __device__ constexpr int recv_entries(int bx, int by, int bz)
{
    return 2 * (by * (bz / 2) + bx * (bz / 2) + bx * by) + 4 * (bx + by + bz / 2);
}

// Kernel kinds for per-kernel timing.
enum KernelKind { K_MACRO = 0, K_ACTIVATE = 1, K_COLLIDE = 2, K_OTHER = 3 };

// The kernels of one storage form (lbm_step.cuh, compiled once per form).
struct StorageOps {
    cudaError_t (*init)(const KParams &, const float *, int, int, int, cudaStream_t);
    cudaError_t (*init_finish)(const KParams &, int, int, cudaStream_t);
    cudaError_t (*ambient_slot)(const KParams &, cudaStream_t);
    cudaError_t (*macro)(const KParams &, int, int, int, cudaStream_t);
    cudaError_t (*activate)(const KParams &, int, int, cudaStream_t);
    cudaError_t (*collide)(const KParams &, int, int, cudaStream_t);
    cudaError_t (*output)(const KParams &, int, int, int, int, float *, int, cudaStream_t);
    cudaError_t (*mass_partial)(const KParams &, int, int, double *, int, cudaStream_t);
    cudaError_t (*block_pops)(const KParams &, int, int, float *, cudaStream_t);
    cudaError_t (*features)(const KParams &, int, const int *, const int *, const int *, float *, int,
                            cudaStream_t);
    int (*ctas_per_sm)();
    // nsteps whole steps in one cooperative launch
    cudaError_t (*run)(const KParams &, int, int, int, cudaStream_t);
    // between steps: renumber the meshed slots in block order when due
    cudaError_t (*sort)(const KParams &, int, cudaStream_t);
    // the collision of a step and pass 1 of the next in one launch (FP32,
    // two components, A-B only; cudaErrorNotSupported otherwise)
    cudaError_t (*fused)(const KParams &, int, cudaStream_t);
};
const StorageOps *storage_ops_fp32();
const StorageOps *storage_ops_fp32_16x8x4();
const StorageOps *storage_ops_fp32_16x4x8();
const StorageOps *storage_ops_fp32_32x4x4();
const StorageOps *storage_ops_fp16();
const StorageOps *storage_ops_bf16();

// Launch wrappers (lbm_kernels.cu), dispatching on kp.storage.  All enqueue
// on `s` and return the launch status.
// Initial state of slots [slot0, slot0 + nslots) from in_block; once every
// initial slot is done, launch_init_finish (the 16-bit forms write their
// populations there, when all reference densities are known).
cudaError_t launch_init(const KParams &kp, const float *in_block, int slot0, int nslots,
                        int grid, cudaStream_t s);
cudaError_t launch_init_finish(const KParams &kp, int nslots, int sms, cudaStream_t s);
cudaError_t launch_ambient_slot(const KParams &kp, cudaStream_t s);
// The cell kernels size their persistent grids themselves: `sms` x the
// CTAs per SM their occupancy allows.
cudaError_t launch_macro(const KParams &kp, int step, int criterion, int sms, cudaStream_t s);
cudaError_t launch_activate(const KParams &kp, int step, int sms, cudaStream_t s);
cudaError_t launch_collide(const KParams &kp, int step, int sms, cudaStream_t s);
// The collision of the step and pass 1 (with the criterion in progressive
// mode) of the next one, in one launch.
cudaError_t launch_fused(const KParams &kp, int sms, cudaStream_t s);
// Block-order rank r -> block id in the slot order of kp.strip (host and
// device share the definition).
__host__ __device__ inline int strip_block(int r, int nbx, int nby, int nbz, int strip)
{
    if (strip <= 0 || strip >= nby) return r;
    const int full = strip * nbx * nbz;  // blocks of a full strip
    const int k = r / full;
    const int h = (k + 1) * strip <= nby ? strip : nby - k * strip;  // rows of strip k
    const int rr = r - k * full;
    const int z = rr / (nbx * h), rem = rr % (nbx * h);
    return rem % nbx + nbx * (k * strip + rem / nbx + nby * z);
}
cudaError_t launch_output(const KParams &kp, int rd, int comp, int slot0, int nslots, float *out,
                          int sms, cudaStream_t s);
cudaError_t launch_mass(const KParams &kp, int rd, int n, double *partial, double *out, int grid,
                        cudaStream_t s);
// FP32 populations of one slot of buffer rd into out[ncomp][Q][CELLS] (16-bit forms).
cudaError_t launch_sort(const KParams &kp, int sms, cudaStream_t s);
cudaError_t launch_block_pops(const KParams &kp, int rd, int slot, float *out, cudaStream_t s);
// nsteps steps in one cooperative launch with grid barriers between the
// phases (bounded waits: a barrier that does not complete sets
// LBM_ETIMEOUT in the control words).
cudaError_t launch_run(const KParams &kp, int nsteps, int progressive, int sms, cudaStream_t s);
// One grid barrier that expects `missing` more CTAs than are launched, on
// a scratch control block (tests of the bounded wait); returns the status.
int barrier_selftest(int missing, long long spins, int sms);
int max_ctas_per_sm_stream_kernels(int storage);

// Frontier blocks and their features (lbm_kernels.cu; features per storage
// form).  mark/list: [nblocks] scratch, count: one int (zeroed by the
// caller with mark); par: the read buffer; nsnap: a device copy of the
// meshed-block count taken between two steps (only those slots are read).
cudaError_t launch_frontier(const KParams &kp, const int *nsnap, unsigned *mark, int *list, int *count,
                            int sms, cudaStream_t s);
cudaError_t launch_features(const KParams &kp, int par, const int *nsnap, const int *list,
                            const int *count, float *feat, int sms, cudaStream_t s);
// Prepare the listed blocks whose probability exceeds thr (side stream).
cudaError_t launch_prepare(const KParams &kp, const int *list, const int *count, const float *prob,
                           float thr, unsigned *prep, uint32_t *nbits_pre, int sms, cudaStream_t s);
// The network's forward pass on a stream (lbm_mlp.cu); the sample count is
// n, or *ndev when ndev is not NULL.
cudaError_t mlp_forward_on(const lbm_mlp *m, const float *x, int n, const int *ndev, int bf16,
                           float *prob, cudaStream_t s);

// Message returned by lbm_last_error(NULL) (lbm_capi.cpp).
void set_global_error(const char *msg);

}  // namespace lbm
