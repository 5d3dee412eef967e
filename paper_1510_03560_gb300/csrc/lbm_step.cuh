// Device side of liblbm: the progressive-mesh two-component pseudo-potential
// LBM step (arXiv:1510.03560, Sec. 2 and Sec. 4) for sm_103a, written once
// for every storage form of the populations and compiled once per form
// (lbm_kernels.cu: FP32, lbm_kernels_f16.cu: FP16, lbm_kernels_bf16.cu:
// BF16).
//
// Layout in HBM (block-major structure of arrays, Sec. 3: SoA for
// coalescing):
//   f[buf][slot][comp][dir][cell]   populations, two buffers (A-B pattern,
//                                   Sec. 3), cell = x + 8 (y + 8 z); FP32,
//                                   or 16-bit deviations (below)
//   mac[par][slot][cell]            float4 (rho0, rho1, psi0, 0) of the step;
//                                   one copy (FP32) or two by step parity
//   nbits[slot][cell]               bit i: cell x - e_i is solid; bit 19: held
//   uprev[slot][comp][3][cell]      velocity of the previous step, read and
//                                   written only at cells bordering
//                                   unmeshed blocks (criterion, Eq. 13)
// A warp covers four x-rows of one z-plane of a block: every population
// access of a warp touches consecutive sectors of one plane.
//
// 16-bit forms: the value stored at (x, i) is f_i - w_i rho_r, rho_r the
// density at the writing step of the cell that reads it next (x + e_i, or x
// itself when x + e_i is solid).  The writer (the collision) has gathered
// those densities for the forces already; a reader needs only its own
// previous density, one load per cell.  Populations coming from the
// ambient state (unmeshed blocks, blocks created in this step) are the
// ambient equilibrium itself.  Held cells keep their density in mac and
// their velocity in uprev and are rewritten every step.
//
// The step kernels have no block-wide barrier.  A CTA of 256 threads works on
// half a block at a time (grid-stride over half-blocks); every warp fetches
// the slots of the 27 blocks around its block with one lane-parallel load
// and hands them out with shuffles, and reads the per-cell solid bits
// instead of block masks.
//
// One time step is these launches:
//   k_macro    pull streaming + Eqs. 4-5 + Eqs. 6-7 -> mac; criterion of
//              Eq. 13 at cells bordering unmeshed blocks, marking targets;
//              its last CTA renumbers the step's candidates in block order
//   k_activate new blocks: slots, ambient equilibrium, their k_macro work
//   k_collide  pull streaming again + forces (Eqs. 8-9, gravity,
//              adhesion) from the neighbours' mac + forced BGK collision
//              (Eqs. 10-12) -> f of the other buffer
// (or, fused, k_fused2: the collision of a step and k_macro's work for the
// next one in a single launch; or, with the density partials, a collision
// that also sums the next step's densities and a pass 1 split into
// k_macro2p / k_macro2f that adds them; see below)
// Between steps, now and then, the k_sort_* launches renumber the meshed
// slots in the slot order (locality; "slot order" below).  Further sections:
// A-A streaming (one population array, Sec. 3), the TMA-staged and
// deviation-form kernels, the cooperative multi-step kernel.  The file is
// compiled once per storage form and, for FP32, once per block shape.
#pragma once

#include <climits>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// Checked builds (-DLBM_CHECKED) test the slot and block indices of the step
// kernels before use; a failure records the site and value in the control
// words (lbm_step then fails) and the access is skipped.  Normal builds
// compile the checks away.
#ifdef LBM_CHECKED
__device__ __forceinline__ bool in_range(const KParams &kp, long long v, long long hi, int site)
{
    if (v >= 0 && v < hi) return true;
    if (atomicCAS(&kp.ctrl->check_site, 0, site) == 0) kp.ctrl->check_value = v;
    return false;
}
#else
__device__ __forceinline__ bool in_range(const KParams &, long long, long long, int) { return true; }
#endif
// End of a step's collide launch: the last CTA to finish advances the
// device step counter (every CTA read it at its start), so that a captured
// sequence of step launches can be replayed.
__device__ __forceinline__ void step_done(Ctrl *ctrl, int step)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctrl->collide_done, 1u) == gridDim.x - 1) {
            ctrl->collide_done = 0u;
            if (ctrl->status == 0) ctrl->step = step + 1;
            __threadfence();
        }
    }
}

// The candidates of a step renumbered in block order by the last CTA of the
// launch that marked them (defined with order_body below).
__device__ void order_tail(const KParams &kp, int step);

constexpr int THREADS = 256;            // threads per CTA of the cell kernels
// resident CTAs per SM the deviation-form step kernels are compiled for
// (fewer registers would spill)
constexpr int DEV_MACRO_MIN_CTAS = 2;
constexpr int DEV_COLLIDE_MIN_CTAS = 2;
constexpr int PARTS = CELLS / THREADS;  // CTA work items per block

// Stores of a warp cover four 8-cell x-rows, one 32-byte sector per row
// and population.  Every lane of the warp must call (a ballot).  A sector written only in part makes the memory read it
// back to merge (read-modify-write under ECC), so a solid cell writes a
// zero wherever another cell of its row writes: complete sectors.  Rows
// with no writer stay untouched.  Solid cells' values are never read.
__device__ __forceinline__ bool row_has(bool p)
{
    const unsigned m = __ballot_sync(0xffffffffu, p);
    return (m >> ((threadIdx.x & 31) & 24u)) & 0xffu;
}

// ---- D3Q19 in this library's order: the 9 velocities with e_z = 0, then
// the 5 with e_z = +1, then the 5 with e_z = -1; opposites are adjacent
// within the first group and 5 apart across the other two. -------------
__host__ __device__ constexpr int cx(int i)
{
    return (i == 1 || i == 5 || i == 7 || i == 10 || i == 16) ? 1
           : (i == 2 || i == 6 || i == 8 || i == 11 || i == 15) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int cy(int i)
{
    return (i == 3 || i == 5 || i == 8 || i == 12 || i == 18) ? 1
           : (i == 4 || i == 6 || i == 7 || i == 13 || i == 17) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int cz(int i) { return (i >= 9 && i <= 13) ? 1 : (i >= 14 ? -1 : 0); }
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : (i <= 8 ? ((i & 1) ? i + 1 : i - 1) : (i <= 13 ? i + 5 : i - 5));
}
__host__ __device__ constexpr float wgt(int i)
{
    return i == 0 ? 1.0f / 3.0f
                  : ((i <= 4 || i == 9 || i == 14) ? 1.0f / 18.0f : 1.0f / 36.0f);
}
// One representative of each opposite pair, and the representative of any
// moving velocity's pair.
__host__ __device__ constexpr int pair_rep(int p)
{
    return p < 4 ? 1 + 2 * p : 5 + p;  // 1 3 5 7 | 9 10 11 12 13
}
__host__ __device__ constexpr int rep_of(int i)
{
    return i <= 8 ? ((i & 1) ? i : i - 1) : (i <= 13 ? i : i - 5);
}
constexpr int NPAIR = 9;

template <int I, int N>
struct Unroll {
    template <class F>
    __device__ __forceinline__ static void run(F &&f)
    {
        f.template operator()<I>();
        Unroll<I + 1, N>::run(f);
    }
};
template <int N>
struct Unroll<N, N> {
    template <class F>
    __device__ __forceinline__ static void run(F &&) {}
};

// ---- storage forms ----------------------------------------------------------
// FP32: one float per (component, direction, cell).  Deviation forms: one
// 32-bit word per (direction, cell) holding both components' 16-bit
// deviations (component 0 in the low half), so that a warp's access moves
// 128 bytes like the FP32 form's.
template <int ST>
struct Store;
template <>
struct Store<LBM_STORAGE_FP32> {
    using T = float;
    static constexpr bool DEV = false;
};
template <>
struct Store<LBM_STORAGE_FP16> {
    using T = uint32_t;
    static constexpr bool DEV = true;
    __device__ static __forceinline__ float2 dec2(uint32_t w)
    {
        __half2 h;
        __builtin_memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    __device__ static __forceinline__ uint32_t enc2(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        __builtin_memcpy(&w, &h, 4);
        return w;
    }
};
template <>
struct Store<LBM_STORAGE_BF16> {
    using T = uint32_t;
    static constexpr bool DEV = true;
    // a bfloat16 is the upper half of the FP32 with the same value
    __device__ static __forceinline__ float2 dec2(uint32_t w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    __device__ static __forceinline__ uint32_t enc2(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        __builtin_memcpy(&w, &h, 4);
        return w;
    }
};

template <int ST>
__device__ __forceinline__ typename Store<ST>::T *pops(const KParams &kp)
{
    if constexpr (ST == LBM_STORAGE_FP32)
        return kp.f;
    else
        return reinterpret_cast<uint32_t *>(kp.h);
}

// ---- block shape -------------------------------------------------------------
// BX x BY x BZ cells per block (512 in all), cell c = x + BX (y + BY z).  The
// default is 8^3; a translation unit may define LBM_BLOCK_X/Y/Z before
// including this file to compile the kernels for another shape.  x-rows are
// whole 32-byte sectors (BX a multiple of 8), so a warp (32 consecutive
// cells) still reads and writes whole sectors.
#ifndef LBM_BLOCK_X
#define LBM_BLOCK_X 8
#define LBM_BLOCK_Y 8
#define LBM_BLOCK_Z 8
#endif
constexpr int BX = LBM_BLOCK_X, BY = LBM_BLOCK_Y, BZ = LBM_BLOCK_Z;
constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
constexpr int SHX = ilog2(BX), SHXY = ilog2(BX * BY);
static_assert(BX * BY * BZ == CELLS, "a block holds 512 cells");
static_assert((1 << SHX) == BX && (1 << ilog2(BY)) == BY && (1 << ilog2(BZ)) == BZ,
              "block extents are powers of two");
static_assert(BX % 8 == 0 && BY >= 2 && BZ >= 2, "x-rows of whole sectors; a one-cell halo per axis");
__device__ __forceinline__ int lx_of(int c) { return c & (BX - 1); }
__device__ __forceinline__ int ly_of(int c) { return (c >> SHX) & (BY - 1); }
__device__ __forceinline__ int lz_of(int c) { return c >> SHXY; }

// Neighbour-block index (0..26) of a local coordinate in [-1, B].
template <int B>
__device__ __forceinline__ int side(int v) { return v < 0 ? 0 : (v > B - 1 ? 2 : 1); }
__device__ __forceinline__ int nbk(int x, int y, int z) { return side<BX>(x) + 3 * side<BY>(y) + 9 * side<BZ>(z); }
__device__ __forceinline__ int lcell(int x, int y, int z)
{
    return (x & (BX - 1)) | ((y & (BY - 1)) << SHX) | ((z & (BZ - 1)) << SHXY);
}

__device__ __forceinline__ int neighbour_block(const KParams &kp, int x, int y, int z)
{
    if (x < 0 || x >= kp.nbx) {
        if (!kp.per[0]) return -1;
        x = (x + kp.nbx) % kp.nbx;
    }
    if (y < 0 || y >= kp.nby) {
        if (!kp.per[1]) return -1;
        y = (y + kp.nby) % kp.nby;
    }
    if (z < 0 || z >= kp.nbz) {
        if (!kp.per[2]) return -1;
        z = (z + kp.nbz) % kp.nbz;
    }
    return x + kp.nbx * (y + kp.nby * z);
}

__device__ __forceinline__ int neighbour_of(const KParams &kp, int gid, int k)
{
    const int bx = gid % kp.nbx, by = (gid / kp.nbx) % kp.nby, bz = gid / (kp.nbx * kp.nby);
    return neighbour_block(kp, bx + k % 3 - 1, by + (k / 3) % 3 - 1, bz + k / 9 - 1);
}

// The 27 blocks around `gid`, one slot per lane (lane 13: the block itself,
// or unmeshed with own_unmeshed; lanes 27-31: SOLIDBLK), and the
// warp-uniform mask of unmeshed neighbours.  Slots >= slot_limit count as
// unmeshed.  Every lane of the warp calls it.
struct WarpNbr {
    int slot;         // slot, AMBIENT or SOLIDBLK
    unsigned amb;     // warp-uniform: bit k set when neighbour k is unmeshed
    uint32_t fbase;   // population offset of the slot (the ambient slot for
                      // unmeshed or solid blocks)
    uint32_t mbase;   // first-pass value offset in kp.mac, likewise (plus
                      // the offset of the parity in use)
};

__device__ __forceinline__ WarpNbr make_nbr(const KParams &kp, int s, uint32_t moff = 0)
{
    const uint32_t q = s >= 0 ? (uint32_t)s : (uint32_t)kp.amb_slot;
    return WarpNbr{s, __ballot_sync(FULL, s == AMBIENT) & ~(1u << 13), q * (uint32_t)kp.slot_floats,
                   q * (uint32_t)CELLS + moff};
}

__device__ __forceinline__ WarpNbr warp_nbr(const KParams &kp, int gid, int own_slot, int slot_limit,
                                            bool own_unmeshed = false)
{
    const int lane = threadIdx.x & 31;
    int s = SOLIDBLK;
    if (lane == 13) {
        s = own_unmeshed ? AMBIENT : own_slot;
    } else if (lane < 27) {
        const int nid = neighbour_of(kp, gid, lane);
        if (nid >= 0) {
            s = kp.slot_of[nid];
            if (s >= slot_limit) s = AMBIENT;
        }
    }
    return make_nbr(kp, s);
}

// The same, read from the slot's row of the neighbour-slot table (kept up to
// date by block creation): one coalesced 128-byte load per warp.
__device__ __forceinline__ int nbr_row_lane(const KParams &kp, int slot)
{
    return kp.nbr[(size_t)slot * NBR_STRIDE + (threadIdx.x & 31)];
}
__device__ __forceinline__ WarpNbr warp_nbr_of(const KParams &kp, int lane_slot, uint32_t moff = 0)
{
    return make_nbr(kp, lane_slot, moff);
}



// Neighbour blocks reachable from a cell through the 18 moving velocities.
__device__ __forceinline__ unsigned reach_bits(int lx, int ly, int lz)
{
    unsigned r = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) r |= 1u << nbk(lx + cx(i), ly + cy(i), lz + cz(i));
    return r & ~(1u << 13);
}

// Solid / held word of one cell from the per-block masks (bit i: x - e_i is
// solid, cells outside a non-periodic axis are solid; bit HELD_BIT: held).
__device__ uint32_t cell_bits(const KParams &kp, int gid, int c)
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = lx - cx(i), sy = ly - cy(i), sz = lz - cz(i);
        const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
        const int nid = k == 13 ? gid : neighbour_of(kp, gid, k);
        const bool solid =
            nid < 0 || ((kp.solid[(size_t)nid * MASK_WORDS + (lc >> 5)] >> (lc & 31)) & 1u);
        bits |= (uint32_t)solid << i;
    }
    if ((kp.held[(size_t)gid * MASK_WORDS + (c >> 5)] >> (c & 31)) & 1u) bits |= 1u << HELD_BIT;
    return bits;
}

// The same word with the 27 neighbour block ids given one per lane (lane k:
// block k of the 27 around gid, -1 outside a non-periodic axis; lane 13:
// gid), so that no lane recomputes them per direction.  Every lane of the
// warp calls (shuffles).
__device__ __forceinline__ uint32_t cell_bits_nbr(const KParams &kp, int gid, int nid_lane, int c)
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    uint32_t bits = 0;
    Unroll<0, Q>::run([&]<int I>() {
        const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
        const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
        const int nid = __shfl_sync(FULL, nid_lane, k);
        const bool solid =
            nid < 0 || ((kp.solid[(size_t)nid * MASK_WORDS + (lc >> 5)] >> (lc & 31)) & 1u);
        bits |= (uint32_t)solid << I;
    });
    if ((kp.held[(size_t)gid * MASK_WORDS + (c >> 5)] >> (c & 31)) & 1u) bits |= 1u << HELD_BIT;
    return bits;
}

// Source offset (in the read buffer) of the population moving along e_I
// into cell c: from x - e_I; the cell's own opposite population behind a
// solid cell (halfway bounce-back); its own population at held cells.
// `own` is the cell's own offset.  Every lane calls (one shuffle).
template <int I>
__device__ __forceinline__ uint32_t src_offset(const WarpNbr &wn, uint32_t own, int lx, int ly,
                                               int lz, uint32_t bits, bool held, int &k)
{
    const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
    k = nbk(sx, sy, sz);
    const int lc = lcell(sx, sy, sz);
    const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
    const bool bounce = (bits >> I) & 1u;
    return held ? own + (uint32_t)(I * CELLS)
                : (bounce ? own + (uint32_t)(opp(I) * CELLS) : base + (uint32_t)(I * CELLS + lc));
}

// The loads of one cell's pull in a deviation form, issued but not yet
// used: one packed word per direction, and which populations come from
// the ambient state (unmeshed source blocks, or the cell's own block when
// it was created in this step).
struct DevLoad {
    uint32_t v[Q];
    uint32_t ambs;
};

template <int ST>
__device__ __forceinline__ void dev_issue(const KParams &kp, const WarpNbr &wn, const uint32_t *rd,
                                          int own_slot, int c, uint32_t bits, bool live,
                                          bool own_ambient, DevLoad &L)
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    const uint32_t own =
        (own_ambient ? (uint32_t)kp.amb_slot : (uint32_t)own_slot) * (uint32_t)kp.slot_floats + (uint32_t)c;
    const bool held = (bits >> HELD_BIT) & 1u;
    const unsigned ambm = wn.amb | (own_ambient ? (1u << 13) : 0u);
    uint32_t off[Q];
    Unroll<0, Q>::run([&]<int I>() {
        int k;
        off[I] = src_offset<I>(wn, own, lx, ly, lz, bits, held, k);
    });
    // which populations come from the ambient state; none in a warp with
    // no unmeshed neighbour block (most warps: the flags are skipped there)
    uint32_t ambs = 0;
    if (ambm != 0u) {  // warp-uniform
        Unroll<0, Q>::run([&]<int I>() {
            const int k = nbk(lx - cx(I), ly - cy(I), lz - cz(I));
            const bool bounce = (bits >> I) & 1u;
            const bool a = (held || bounce) ? own_ambient : ((ambm >> k) & 1u);
            ambs |= (uint32_t)a << I;
        });
    }
    L.ambs = ambs;
    Unroll<0, Q>::run([&]<int I>() { L.v[I] = live ? __ldg(rd + off[I]) : 0u; });
}

// Decode the loads of dev_issue: the FP32 populations are the stored
// deviations plus w_I rho_prev (the cell's own previous density `ref`), or
// plus the ambient equilibrium for ambient sources; sink(a, I, f) in pull
// order.
template <int NC, int ST, class Sink>
__device__ __forceinline__ void dev_consume(const KParams &kp, const DevLoad &L, const float ref[2],
                                            Sink &&sink)
{
    auto one = [&]<int I>() {
        const float2 x = Store<ST>::dec2(L.v[I]);
        const bool amb = (L.ambs >> I) & 1u;
        sink.template operator()<I>(0, amb ? kp.famb[0][I] + x.x : __fmaf_rn(wgt(I), ref[0], x.x));
        if constexpr (NC == 2)
            sink.template operator()<I>(1, amb ? kp.famb[1][I] + x.y : __fmaf_rn(wgt(I), ref[1], x.y));
    };
    one.template operator()<0>();
    Unroll<0, NPAIR>::run([&]<int P>() {
        one.template operator()<pair_rep(P)>();
        one.template operator()<opp(pair_rep(P))>();
    });
}

// Pull streaming (Eq. 10, left-hand side) of every component of one cell,
// rest first, then opposite pairs, handing each arriving population to
// sink(a, I, v).  The population moving along e_I comes from x - e_I:
// halfway bounce-back when that cell is solid, the ambient resting
// population when its block is unmeshed, the stored value otherwise; held
// cells keep their own.  With own_ambient the cell's own block is one created
// in this step, still at the ambient state, and is not read back.  In the
// deviation forms `ref` is the cell's own density of the previous step
// (the reference its incoming values were written against) and held cells'
// values are not meaningful.  All lanes must call (shuffles); `live` masks
// the loads.
template <int NC, int ST, class Sink>
__device__ __forceinline__ void pull(const KParams &kp, const WarpNbr &wn,
                                     const typename Store<ST>::T *rd, int own_slot, int c, int lx,
                                     int ly, int lz, uint32_t bits, bool live, bool own_ambient,
                                     const float ref[2], Sink &&sink)
{
    if constexpr (Store<ST>::DEV) {
        DevLoad L;
        dev_issue<ST>(kp, wn, rd, own_slot, c, bits, live, own_ambient, L);
        dev_consume<NC, ST>(kp, L, ref, sink);
    } else {
        const uint32_t own = (own_ambient ? (uint32_t)kp.amb_slot : (uint32_t)own_slot) *
                                 (uint32_t)kp.slot_floats + (uint32_t)c;
        const bool held = (bits >> HELD_BIT) & 1u;
        // Three phases, so that all of a cell's loads are in flight together:
        // (1) the source offset of every population (32-bit, from the read
        // buffer; one shuffle each: unmeshed blocks read the ambient slot),
        // (2) every load, (3) the sink.
        uint32_t off[Q];
        Unroll<0, Q>::run([&]<int I>() {
            const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
            const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
            const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
            const bool bounce = (bits >> I) & 1u;
            off[I] = held ? own + (uint32_t)(I * CELLS)
                          : (bounce ? own + (uint32_t)(opp(I) * CELLS) : base + (uint32_t)(I * CELLS + lc));
        });
        float v[NC][Q];
        Unroll<0, Q>::run([&]<int I>() {
#pragma unroll
            for (int c2 = 0; c2 < NC; ++c2) v[c2][I] = live ? __ldg(rd + off[I] + c2 * Q * CELLS) : 0.f;
        });
        auto one = [&]<int I>() {
#pragma unroll
            for (int c2 = 0; c2 < NC; ++c2) sink.template operator()<I>(c2, v[c2][I]);
        };
        one.template operator()<0>();
        Unroll<0, NPAIR>::run([&]<int P>() {
            one.template operator()<pair_rep(P)>();
            one.template operator()<opp(pair_rep(P))>();
        });
    }
}

// Load of a population.  CG: through L2 only (ld.global.cg), for values
// written earlier in the same launch by other CTAs (the fused step); else
// through the read-only path.
template <bool CG>
__device__ __forceinline__ float ldpop(const float *p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return __ldg(p);
}

// pull() of the FP32 form for two components, handing both components of
// each direction to sink(I, (f_0, f_1)) together.
// mid() runs between issuing the loads and the first sink (work that can
// overlap their latency).
struct NoMid {
    __device__ __forceinline__ void operator()() const {}
};
template <bool CG = false, class Sink, class Mid = NoMid>
__device__ __forceinline__ void pull2_f32(const KParams &kp, const WarpNbr &wn, const float *rd,
                                          int own_slot, int c, int lx, int ly, int lz, uint32_t bits,
                                          bool live, Sink &&sink, Mid &&mid = Mid{})
{
    const uint32_t own = (uint32_t)own_slot * (uint32_t)kp.slot_floats + (uint32_t)c;
    const bool held = (bits >> HELD_BIT) & 1u;
    uint32_t off[Q];
    Unroll<0, Q>::run([&]<int I>() {
        const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
        const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
        const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
        const bool bounce = (bits >> I) & 1u;
        off[I] = held ? own + (uint32_t)(I * CELLS)
                      : (bounce ? own + (uint32_t)(opp(I) * CELLS) : base + (uint32_t)(I * CELLS + lc));
    });
    float2 v[Q];
    Unroll<0, Q>::run([&]<int I>() {
        v[I] = live ? make_float2(ldpop<CG>(rd + off[I]), ldpop<CG>(rd + off[I] + Q * CELLS))
                    : make_float2(0.f, 0.f);
    });
    mid();
    sink.template operator()<0>(v[0]);
    Unroll<0, NPAIR>::run([&]<int P>() {
        sink.template operator()<pair_rep(P)>(v[pair_rep(P)]);
        sink.template operator()<opp(pair_rep(P))>(v[opp(pair_rep(P))]);
    });
}

// Deviation forms: the reference density of each population a cell writes,
// the previous-step density of the cell that reads it (rd[a][i]; the cell
// itself for the rest population and behind solid cells), from `mac`.
// Unmeshed readers give the ambient values (the ambient slot).  All lanes
// must call; `gather` masks the loads.
template <int NC>
__device__ __forceinline__ void reader_refs(const WarpNbr &wn, const float4 *mac, int lx, int ly,
                                            int lz, uint32_t bits, bool gather, const float own[2],
                                            float rdst[2][Q])
{
#pragma unroll
    for (int a = 0; a < NC; ++a) rdst[a][0] = own[a];
    Unroll<1, Q>::run([&]<int D>() {
        const int tx = lx + cx(D), ty = ly + cy(D), tz = lz + cz(D);
        const int k = nbk(tx, ty, tz), lc = lcell(tx, ty, tz);
        const uint32_t mb = __shfl_sync(FULL, wn.mbase, k);
        const bool solid_n = (bits >> opp(D)) & 1u;  // x + e_D = x - e_opp(D)
        const float4 m = gather ? __ldg(mac + mb + lc) : make_float4(0.f, 0.f, 0.f, 0.f);
        rdst[0][D] = solid_n ? own[0] : m.x;
        if (NC == 2) rdst[1][D] = solid_n ? own[1] : m.y;
    });
}

// Eqs. 4-5 accumulated in pull order: the density as a running sum, the
// momentum from each opposite pair's difference.
struct Moments {
    float rho[2] = {0.f, 0.f};
    float j[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float first[2] = {0.f, 0.f};
    template <int I>
    __device__ __forceinline__ void add(int a, float v)
    {
        rho[a] += v;
        if constexpr (I == 0) {
            return;
        } else if constexpr (rep_of(I) == I) {
            first[a] = v;
        } else {
            constexpr int R = rep_of(I);
            const float d = first[a] - v;
            if (cx(R) > 0) j[a][0] += d; else if (cx(R) < 0) j[a][0] -= d;
            if (cy(R) > 0) j[a][1] += d; else if (cy(R) < 0) j[a][1] -= d;
            if (cz(R) > 0) j[a][2] += d; else if (cz(R) < 0) j[a][2] -= d;
        }
    }
};

// ---- component pairs --------------------------------------------------------
// The two components' values side by side in a float2, computed with the
// paired FP32 instructions of sm_100 and later: one instruction, two
// results, each rounded as the scalar operation would be.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sel2(bool p, float2 a, float2 b) { return p ? a : b; }

// Weight class of a velocity: 0 rest, 1 axis, 2 diagonal.
__host__ __device__ constexpr int wclass(int i)
{
    return i == 0 ? 0 : ((i <= 4 || i == 9 || i == 14) ? 1 : 2);
}

// Eqs. 4-5 for both components at once, in the order of Moments.
struct Moments2 {
    float2 rho = {0.f, 0.f};
    float2 j[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float2 first = {0.f, 0.f};
    template <int I>
    __device__ __forceinline__ void add(float2 v)
    {
        rho = add2(rho, v);
        if constexpr (I == 0) {
            return;
        } else if constexpr (rep_of(I) == I) {
            first = v;
        } else {
            constexpr int R = rep_of(I);
            const float2 d = sub2(first, v);
            if (cx(R) > 0) j[0] = add2(j[0], d); else if (cx(R) < 0) j[0] = sub2(j[0], d);
            if (cy(R) > 0) j[1] = add2(j[1], d); else if (cy(R) < 0) j[1] = sub2(j[1], d);
            if (cz(R) > 0) j[2] = add2(j[2], d); else if (cz(R) < 0) j[2] = sub2(j[2], d);
        }
    }
};

// dev_consume for both components at once: each population is the decoded
// deviation plus w_I rho_prev (wref, by weight class) or plus the ambient
// equilibrium (famb, by weight class) for ambient sources.
template <int ST, class Sink>
__device__ __forceinline__ void dev_consume2(const DevLoad &L, const float2 wref[3],
                                             const float2 famb[3], Sink &&sink)
{
    auto all = [&](auto amb_of) {
        auto one = [&]<int I>() {
            const float2 x = Store<ST>::dec2(L.v[I]);
            sink.template operator()<I>(add2(x, sel2(amb_of(I), famb[wclass(I)], wref[wclass(I)])));
        };
        one.template operator()<0>();
        Unroll<0, NPAIR>::run([&]<int P>() {
            one.template operator()<pair_rep(P)>();
            one.template operator()<opp(pair_rep(P))>();
        });
    };
    // warp-uniform: most warps have no ambient source, and skip the selects
    if (__any_sync(FULL, L.ambs != 0u))
        all([&](int i) { return ((L.ambs >> i) & 1u) != 0u; });
    else
        all([](int) { return false; });
}

// ---- A-A streaming: addressing (FP32, two components) ----------------------
// One population array updated in place (the A-A pattern of Sec. 3).  Step t
// is a neighbour step when t is even and a local step when t is odd:
//   neighbour step: the population arriving at x along e_i is read at
//     (x - e_i, slot opp(i)); the value leaving x along e_i is written to
//     (x + e_i, slot i);
//   local step: read at (x, slot i), written to (x, slot opp(i)).
// In a step every location is read and written by one cell only, so the
// update is in place.  Halfway bounce-back: a neighbour step reads (x, i)
// when x - e_i is solid and writes (x, opp(i)) when x + e_i is solid; a
// local step needs no case.  Unmeshed source blocks give the ambient
// equilibrium (the ambient slot).  A neighbour step's value leaving towards
// an unmeshed block is parked at (x, opp(i)), a location no other cell
// reads or writes in that step.  A block created in a local step takes the
// parked values of its meshed neighbours as its incoming populations (the
// values the A-B pull reads from their buffers); one created in a neighbour
// step starts from the ambient equilibrium in every slot.  In a local step's
// collision, blocks created in the same step are ambient sources (their
// slots now hold their own incoming values).  Held cells keep their
// constant populations in held_f and write them like any other cell.  The
// initial state is laid out as after a local step: f_i(x) at (x, opp(i)).
// The values and the arithmetic order are those of the A-B kernels, so the
// results are the same bit for bit.

// Offset (component 0; component 1 is Q * CELLS further) of the population
// arriving along e_I at the cell (lx, ly, lz) in an A-A step.  own = slot *
// slot_floats + c, amb_own = amb_slot * slot_floats + c; fresh: the
// warp-uniform mask of neighbour blocks created in this step (the
// collision of a local step).  Every lane calls (a shuffle in neighbour
// steps).
template <bool LOCAL, int I>
__device__ __forceinline__ uint32_t aa_src(const WarpNbr &wn, uint32_t own, uint32_t amb_own, int lx,
                                           int ly, int lz, uint32_t bits, unsigned fresh)
{
    const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
    const int k = nbk(sx, sy, sz);
    const bool solid = (bits >> I) & 1u;
    if constexpr (LOCAL) {
        const bool ambient = !solid && (((wn.amb | fresh) >> k) & 1u);
        return (ambient ? amb_own : own) + (uint32_t)(I * CELLS);
    } else {
        const int lc = lcell(sx, sy, sz);
        const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
        return solid ? own + (uint32_t)(I * CELLS) : base + (uint32_t)(opp(I) * CELLS + lc);
    }
}

// Offset of the location that receives the value leaving the cell along e_I
// in an A-A step.  Every lane calls (a shuffle in neighbour steps).
template <bool LOCAL, int I>
__device__ __forceinline__ uint32_t aa_dst(const WarpNbr &wn, uint32_t own, int lx, int ly, int lz,
                                           uint32_t bits)
{
    if constexpr (LOCAL || I == 0) {
        return own + (uint32_t)(opp(I) * CELLS);
    } else {
        const int tx = lx + cx(I), ty = ly + cy(I), tz = lz + cz(I);
        const int k = nbk(tx, ty, tz), lc = lcell(tx, ty, tz);
        const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
        const bool park = ((bits >> opp(I)) & 1u) || ((wn.amb >> k) & 1u);
        return park ? own + (uint32_t)(opp(I) * CELLS) : base + (uint32_t)(I * CELLS + lc);
    }
}

// The pull of one cell in an A-A step, handing both components of each
// direction to sink(I, (f_0, f_1)) in pull2_f32's order.  Held cells read
// their constants.  All lanes call; `live` masks the loads.
template <bool LOCAL, class Sink>
__device__ __forceinline__ void pull2_aa(const KParams &kp, const WarpNbr &wn, int own_slot, int c, int lx,
                                         int ly, int lz, uint32_t bits, bool live, unsigned fresh, Sink &&sink)
{
    const bool held = (bits >> HELD_BIT) & 1u;
    const uint32_t own = (uint32_t)own_slot * (uint32_t)kp.slot_floats + (uint32_t)c;
    const uint32_t amb_own = (uint32_t)kp.amb_slot * (uint32_t)kp.slot_floats + (uint32_t)c;
    const float *src = kp.f;
    uint32_t hown = 0;
    if (held && live) {
        src = kp.held_f;
        hown = (uint32_t)kp.held_rank[kp.block_of[own_slot]] * (uint32_t)kp.slot_floats + (uint32_t)c;
    }
    uint32_t off[Q];
    Unroll<0, Q>::run([&]<int I>() {
        const uint32_t o = aa_src<LOCAL, I>(wn, own, amb_own, lx, ly, lz, bits, fresh);
        off[I] = held ? hown + (uint32_t)(I * CELLS) : o;
    });
    float2 v[Q];
    Unroll<0, Q>::run([&]<int I>() {
        v[I] = live ? make_float2(__ldg(src + off[I]), __ldg(src + off[I] + Q * CELLS))
                    : make_float2(0.f, 0.f);
    });
    sink.template operator()<0>(v[0]);
    Unroll<0, NPAIR>::run([&]<int P>() {
        sink.template operator()<pair_rep(P)>(v[pair_rep(P)]);
        sink.template operator()<opp(pair_rep(P))>(v[opp(pair_rep(P))]);
    });
}

// pull() of the state a reader sees before the step of parity `par`, in the
// A-A layout when the context streams that way (FP32, two components).
template <int NC, int ST, class Sink>
__device__ __forceinline__ void pull_state(const KParams &kp, const WarpNbr &wn,
                                           const typename Store<ST>::T *rd, int par, int slot, int c,
                                           int lx, int ly, int lz, uint32_t bits, bool live,
                                           const float ref[2], Sink &&sink)
{
    if constexpr (!Store<ST>::DEV && NC == 2) {
        if (kp.aa) {
            auto two = [&]<int I>(float2 v) {
                sink.template operator()<I>(0, v.x);
                sink.template operator()<I>(1, v.y);
            };
            if (par)
                pull2_aa<true>(kp, wn, slot, c, lx, ly, lz, bits, live, 0u, two);
            else
                pull2_aa<false>(kp, wn, slot, c, lx, ly, lz, bits, live, 0u, two);
            return;
        }
    }
    pull<NC, ST>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false, ref, sink);
}

// First-pass values of a cell as stored in mac: (rho0, rho1, psi0, 0), so
// that the two densities form one 8-byte pair.
__device__ __forceinline__ float4 mac_pack(float rho0, float psi0, float rho1)
{
    return make_float4(rho0, rho1, psi0, 0.f);
}

// Eq. 7 (Peng-Robinson) and Eq. 6 (pseudo-potential), FP32.
__device__ __forceinline__ float psi_of(const KParams &kp, float rho)
{
    if (kp.g_self == 0.f) return 0.f;
    const float b = kp.pr_b;
    const float p = rho * kp.pr_RT / (1.f - b * rho) -
                    kp.pr_atheta * rho * rho / (1.f + 2.f * b * rho - b * b * rho * rho);
    const float arg = kp.psi_scale * (p - rho * (1.0f / 3.0f));
    return sqrtf(fmaxf(arg, 0.f));
}

// Eq. 2 with c_s^2 = 1/3.
template <int I>
__device__ __forceinline__ float feq(float wrho, float ux, float uy, float uz, float uu)
{
    float eu = 0.f;
    if (cx(I) > 0) eu += ux; else if (cx(I) < 0) eu -= ux;
    if (cy(I) > 0) eu += uy; else if (cy(I) < 0) eu -= uy;
    if (cz(I) > 0) eu += uz; else if (cz(I) < 0) eu -= uz;
    return wrho * (1.f + 3.f * eu + 4.5f * eu * eu - 1.5f * uu);
}

// ---------------------------------------------------------------------------
// Initial state: equilibrium of the initial fields in both buffers, the
// initial velocity as the "previous" one, the cells' solid words.  The
// deviation forms write the densities (mac of parity 1, the reference of
// step 0's reads) and velocities here and the populations in k_init_dev,
// once every initial block's density is known.
// in: [slot - slot0][ncomp][4][CELLS] (rho, ux, uy, uz), block-major.
template <int ST>
__global__ void __launch_bounds__(CELLS) k_init(KParams kp, const float *in, int slot0, int nslots)
{
    using S = Store<ST>;
    const int c = threadIdx.x;
    for (int r = blockIdx.x; r < nslots; r += gridDim.x) {
        const int slot = slot0 + r;
        const int gid = kp.block_of[slot];
        const uint32_t bits = cell_bits(kp, gid, c);
        kp.nbits[(size_t)slot * CELLS + c] = bits;
        const bool solid = bits & 1u;
        const unsigned fluid = __ballot_sync(FULL, !solid && !((bits >> HELD_BIT) & 1u));
        if ((c & 31) == 0 && fluid)
            atomicAdd(&kp.ctrl->fluid_active, (unsigned long long)__popc(fluid));
        float rho_c[2] = {0.f, 0.f};
        for (int a = 0; a < kp.ncomp; ++a) {
            const float *src = in + ((size_t)r * kp.ncomp + a) * 4 * CELLS;
            float rho = src[c], ux = src[CELLS + c], uy = src[2 * CELLS + c],
                  uz = src[3 * CELLS + c];
            if (solid) rho = ux = uy = uz = 0.f;
            rho_c[a] = rho;
            if constexpr (!S::DEV) {
                const float uu = ux * ux + uy * uy + uz * uz;
                float *d0 = kp.f + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
                float *d1 = d0 + kp.buf_stride;
                // A-A: laid out as after a local step, held cells' constants in held_f
                float *hc = kp.aa && ((bits >> HELD_BIT) & 1u)
                                ? kp.held_f + (size_t)kp.held_rank[gid] * kp.slot_floats + a * Q * CELLS + c
                                : nullptr;
                Unroll<0, Q>::run([&]<int I>() {
                    const float v = feq<I>(wgt(I) * rho, ux, uy, uz, uu);
                    if (kp.aa) {
                        d0[opp(I) * CELLS] = v;
                        if (hc) hc[I * CELLS] = v;
                    } else {
                        d0[I * CELLS] = v;
                        d1[I * CELLS] = v;
                    }
                });
            }
            if (kp.uprev) {
                float *up = kp.uprev + ((size_t)slot * kp.ncomp + a) * 3 * CELLS + c;
                up[0] = ux;
                up[CELLS] = uy;
                up[2 * CELLS] = uz;
            }
        }
        if constexpr (S::DEV)
            kp.mac[kp.mac_stride + (size_t)slot * CELLS + c] =
                solid ? make_float4(0.f, 0.f, 0.f, 0.f) : mac_pack(rho_c[0], psi_of(kp, rho_c[0]), rho_c[1]);
    }
}

// Deviation forms: the populations of buffer 0 for the initial slots, the
// equilibrium of (mac[1], uprev) written against the reading cells'
// densities, the rest population from the mass balance.
template <int NC, int ST>
__global__ void __launch_bounds__(THREADS) k_init_dev(KParams kp, int nslots)
{
    using S = Store<ST>;
    const float4 *ref = kp.mac + kp.mac_stride;
    typename S::T *d_all = pops<ST>(kp);
    for (int it = blockIdx.x; it < nslots * PARTS; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
        const bool live = !(bits & 1u);
        const float4 m = __ldg(ref + (size_t)slot * CELLS + c);
        const float own[2] = {m.x, m.y};
        float rdst[2][Q];
        reader_refs<NC>(wn, ref, lx, ly, lz, bits, live, own, rdst);
        uint32_t *dst = d_all + (size_t)slot * kp.slot_floats + c;
        if (!live) {
#pragma unroll
            for (int i = 0; i < Q; ++i) dst[i * CELLS] = 0u;
            continue;
        }
        float ux[2], uy[2], uz[2], uu[2], moving[2] = {0.f, 0.f};
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
            ux[a] = up[0];
            uy[a] = up[CELLS];
            uz[a] = up[2 * CELLS];
            uu[a] = ux[a] * ux[a] + uy[a] * uy[a] + uz[a] * uz[a];
        }
        Unroll<1, Q>::run([&]<int I>() {
            float d[2] = {0.f, 0.f};
#pragma unroll
            for (int a = 0; a < NC; ++a)
                d[a] = __fmaf_rn(-wgt(I), rdst[a][I], feq<I>(wgt(I) * own[a], ux[a], uy[a], uz[a], uu[a]));
            const uint32_t h = S::enc2(d[0], d[1]);
            dst[I * CELLS] = h;
            const float2 back = S::dec2(h);
            moving[0] += __fmaf_rn(wgt(I), rdst[0][I], back.x);
            moving[1] += __fmaf_rn(wgt(I), rdst[1][I], back.y);
        });
        dst[0] = S::enc2(__fmaf_rn(-wgt(0), own[0], own[0] - moving[0]),
                         NC == 2 ? __fmaf_rn(-wgt(0), own[1], own[1] - moving[1]) : 0.f);
    }
}

// The ambient slot: resting ambient populations in both buffers (zero
// deviations in the 16-bit forms) and the ambient first-pass values, read
// wherever a neighbour block is unmeshed.
template <int ST>
__global__ void __launch_bounds__(CELLS) k_ambient_slot(KParams kp)
{
    using S = Store<ST>;
    const int c = threadIdx.x;
    const float psi = psi_of(kp, kp.rho_amb[0]);
    if (c == 0) kp.ctrl->psi_amb = psi;
    typename S::T *base = pops<ST>(kp) + (size_t)kp.amb_slot * kp.slot_floats + c;
    for (int i = 0; i < kp.slot_floats / CELLS; ++i) {
        typename S::T v{};
        if constexpr (!S::DEV) v = kp.famb[i / Q][i % Q];
        base[i * CELLS] = v;
        base[kp.buf_stride + i * CELLS] = v;
    }
    const float4 m = mac_pack(kp.rho_amb[0], psi, kp.rho_amb[1]);
    kp.mac[(size_t)kp.amb_slot * CELLS + c] = m;
    kp.mac[kp.mac_stride + (size_t)kp.amb_slot * CELLS + c] = m;
}

// Streaming + moments of one cell; writes mac (live cells), returns rho and
// the bare velocity.  In the deviation forms `ref` is the cell's previous
// density and a held cell's mac stays `prev`.  All lanes must call.
template <int NC, int ST>
__device__ __forceinline__ void macro_cell(const KParams &kp, const WarpNbr &wn,
                                           const typename Store<ST>::T *rd, float4 *mac, int slot,
                                           int c, int lx, int ly, int lz, uint32_t bits, bool live,
                                           bool own_ambient, const float ref[2], float4 prev,
                                           float rho[2], float u[2][3])
{
    Moments m;
    pull<NC, ST>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, own_ambient, ref,
                 [&]<int I>(int a, float v) { m.template add<I>(a, v); });
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        rho[a] = m.rho[a];
        const float inv = 1.f / m.rho[a];
        u[a][0] = m.j[a][0] * inv;
        u[a][1] = m.j[a][1] * inv;
        u[a][2] = m.j[a][2] * inv;
    }
    if (live) {
        float4 out = mac_pack(rho[0], psi_of(kp, rho[0]), NC == 2 ? rho[1] : 0.f);
        if constexpr (Store<ST>::DEV)
            if ((bits >> HELD_BIT) & 1u) out = prev;
        mac[(size_t)slot * CELLS + c] = out;
    }
}

// Eq. 13 at a fluid cell bordering unmeshed blocks: when the velocity of a
// component changed by more than S since the previous step, the unmeshed
// blocks next to the cell become candidates.  Warp-collective.  CG: the
// previous velocity was written in the same launch (fused step).
template <int NC, bool CG = false>
__device__ __forceinline__ void criterion_mark(const KParams &kp, Ctrl *ctrl, int par, int n, int slot,
                                               int c, const WarpNbr &wn, bool fluid,
                                               const float u[2][3])
{
    const int lane = threadIdx.x & 31;
    const unsigned front = reach_bits(lx_of(c), ly_of(c), lz_of(c)) & wn.amb;
    unsigned tgt = 0;
    if (fluid && front) {
        float d2max = 0.f;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
            float p0, p1, p2;
            if constexpr (CG) {
                p0 = __ldcg(up);
                p1 = __ldcg(up + CELLS);
                p2 = __ldcg(up + 2 * CELLS);
            } else {
                p0 = up[0];
                p1 = up[CELLS];
                p2 = up[2 * CELLS];
            }
            const float dx = u[a][0] - p0, dy = u[a][1] - p1, dz = u[a][2] - p2;
            d2max = fmaxf(d2max, dx * dx + dy * dy + dz * dz);
        }
        if (d2max > kp.S2) tgt = front;
    }
    tgt = __reduce_or_sync(FULL, tgt);
    if (tgt && lane < 27 && ((tgt >> lane) & 1u)) {
        // a candidate takes the next slot after the meshed ones now
        // (k_activate checks the capacity and undoes it if full)
        const int nid = neighbour_of(kp, kp.block_of[slot], lane);
        if (in_range(kp, nid, (long long)kp.nbx * kp.nby * kp.nbz, 3) &&
            atomicCAS(&kp.cand_mark[nid], 0u, 1u) == 0u) {
            const int pos = atomicAdd(&ctrl->ncand[par], 1);
            kp.cand_list[pos] = nid;
            if (n + pos < kp.capacity) kp.slot_of[nid] = n + pos;
        }
    }
}

// Pass 1 of a step (FP32 form): streaming and moments over the meshed
// blocks; with `criterion`, Eq. 13 at fluid cells bordering unmeshed blocks.
template <int NC>
__device__ __forceinline__ void macro_body(const KParams &kp, int step, int criterion)
{
    constexpr int ST = LBM_STORAGE_FP32;
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    const int total = n * PARTS;
    // the neighbour row and solid word of the next item are fetched while
    // the current one is processed
    int it = blockIdx.x;
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, next_row);
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        const bool live = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        // (warp-uniform: the pull below shuffles)
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 2))) continue;
        const float ref[2] = {0.f, 0.f};
        if (!criterion || wn.amb == 0u) {
            // warp-uniform: nothing for the criterion to test, only the
            // densities are needed (summed in the order of Moments)
            float r[2] = {0.f, 0.f};
            pull<NC, ST>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false, ref,
                         [&]<int I>(int a, float v) { r[a] += v; });
            if (live) kp.mac[(size_t)slot * CELLS + c] = mac_pack(r[0], psi_of(kp, r[0]), NC == 2 ? r[1] : 0.f);
            continue;
        }
        float rho[2], u[2][3];
        macro_cell<NC, ST>(kp, wn, rd, kp.mac, slot, c, lx, ly, lz, bits, live, false, ref,
                           make_float4(0.f, 0.f, 0.f, 0.f), rho, u);
        if (criterion) criterion_mark<NC>(kp, ctrl, par, n, slot, c, wn, live && !held, u);
    }
}

template <int NC>
__global__ void __launch_bounds__(THREADS) k_macro(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    macro_body<NC>(kp, step, criterion);
    if (criterion) order_tail(kp, step);
}

// Per weight class: w rho_prev (the references of a cell's incoming values)
// and the ambient equilibrium w rho_amb (the values of ambient sources).
__device__ __forceinline__ void amb_and_refs(const KParams &kp, float2 ref, float2 wref[3],
                                             float2 famb[3])
{
    Unroll<0, 3>::run([&]<int K>() {
        constexpr int I = K == 0 ? 0 : (K == 1 ? 1 : 5);
        wref[K] = mul2(splat(wgt(I)), ref);
        famb[K] = make_float2(kp.famb[0][I], kp.famb[1][I]);
    });
}

// Work items of the deviation-form kernels, software-pipelined: the next
// item's population loads are issued before the current item is processed,
// so that they are in flight during its arithmetic.
struct DevItem {
    int slot, c;
    bool ok;          // warp-uniform: the item's table entries passed the checks
    uint32_t bits;
    WarpNbr wn;
    DevLoad L;
    float2 ref;       // the cell's previous densities (mac of the other parity)
};

template <int ST>
__device__ __forceinline__ void dev_item(const KParams &kp, const uint32_t *rd, const float4 *mac_prev,
                                         int it, int row, uint32_t bits, uint32_t moff, DevItem &d)
{
    d.slot = it / PARTS;
    d.c = (it % PARTS) * THREADS + threadIdx.x;
    d.bits = bits;
    d.wn = warp_nbr_of(kp, row, moff);
    d.ok = __all_sync(FULL, in_range(kp, d.wn.slot + 2, (long long)kp.capacity + 2, 2));
    const bool nonsolid = !(bits & 1u);
    const bool held = (bits >> HELD_BIT) & 1u;
    dev_issue<ST>(kp, d.wn, rd, d.slot, d.c, bits, d.ok && nonsolid && !held, false, d.L);
    d.ref = make_float2(0.f, 0.f);
    if (d.ok && nonsolid) d.ref = __ldg(reinterpret_cast<const float2 *>(mac_prev + (size_t)d.slot * CELLS + d.c));
}

// Pass 1 of a step in the deviation forms (as k_macro).  Held cells keep
// their density: mac of this step is a copy of the previous one.
template <int NC, int ST>
__device__ __forceinline__ void macro_dev_body(const KParams &kp, int step, int criterion)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const uint32_t *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
    float4 *mac = kp.mac + (size_t)par * kp.mac_stride;
    const float4 *mac_prev = kp.mac + (size_t)(par ^ 1) * kp.mac_stride;
    const int total = n * PARTS;
    const int G = gridDim.x;
    int it = blockIdx.x;
    if (it >= total) return;
    DevItem cur;
    dev_item<ST>(kp, rd, mac_prev, it, nbr_row_lane(kp, it / PARTS),
                 kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x], 0u, cur);
    int it2 = it + G;
    int row2 = it2 < total ? nbr_row_lane(kp, it2 / PARTS) : SOLIDBLK;
    uint32_t bits2 =
        it2 < total ? kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += G) {
        DevItem nxt;
        if (it2 < total) {
            dev_item<ST>(kp, rd, mac_prev, it2, row2, bits2, 0u, nxt);
            const int it3 = it2 + G;
            if (it3 < total) {
                row2 = nbr_row_lane(kp, it3 / PARTS);
                bits2 = kp.nbits[(size_t)(it3 / PARTS) * CELLS + (it3 % PARTS) * THREADS + threadIdx.x];
            }
        }
        // (every lane votes: the collective must not sit behind &&)
        const bool any_cell = __any_sync(FULL, !(cur.bits & 1u));
        if (cur.ok && any_cell) {  // skip warps of solid cells only
            const bool live = !(cur.bits & 1u);
            const bool held = (cur.bits >> HELD_BIT) & 1u;
            float2 wref[3], famb[3];
            amb_and_refs(kp, cur.ref, wref, famb);
            if (!criterion || cur.wn.amb == 0u) {
                // warp-uniform: nothing for the criterion to test, only the
                // densities are needed (summed in the order of Moments2)
                float2 rho = make_float2(0.f, 0.f);
                dev_consume2<ST>(cur.L, wref, famb, [&]<int I>(float2 v) { rho = add2(rho, v); });
                if (live)
                    mac[(size_t)cur.slot * CELLS + cur.c] =
                        held ? mac_pack(cur.ref.x, psi_of(kp, cur.ref.x), cur.ref.y)
                             : mac_pack(rho.x, psi_of(kp, rho.x), NC == 2 ? rho.y : 0.f);
                cur = nxt;
                it2 += G;
                continue;
            }
            Moments2 m;
            dev_consume2<ST>(cur.L, wref, famb, [&]<int I>(float2 v) { m.template add<I>(v); });
            const float2 inv = make_float2(1.f / m.rho.x, 1.f / m.rho.y);
            float u[2][3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float2 ud = mul2(m.j[d], inv);
                u[0][d] = ud.x;
                u[1][d] = ud.y;
            }
            if (live)
                mac[(size_t)cur.slot * CELLS + cur.c] =
                    held ? mac_pack(cur.ref.x, psi_of(kp, cur.ref.x), cur.ref.y)
                         : mac_pack(m.rho.x, psi_of(kp, m.rho.x), NC == 2 ? m.rho.y : 0.f);
            if (criterion) criterion_mark<NC>(kp, ctrl, par, n, cur.slot, cur.c, cur.wn, live && !held, u);
        }
        cur = nxt;
        it2 += G;
    }
}

template <int NC, int ST>
__global__ void __launch_bounds__(THREADS, DEV_MACRO_MIN_CTAS) k_macro_dev(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    macro_dev_body<NC, ST>(kp, step, criterion);
    if (criterion) order_tail(kp, step);
}

// Ranks in ascending block order of the blocks b < nb with pick(b), by a
// prefix scan in tiles of 32 blocks per thread: a thread gets its 32
// consecutive flags as a bit mask (warp ballots over coalesced rows), a
// warp-shuffle scan and a scan of the warp totals give its first rank, and
// emit(b, rank) runs for its picked blocks; a running total carries the ranks
// from tile to tile.  Every thread of the CTA must call.
template <class Pick, class Emit>
__device__ __forceinline__ void scan_blocks(int nb, Pick &&pick, Emit &&emit)
{
    constexpr int W = 32;  // flags per thread and tile
    __shared__ int warp_sum[32];
    const int T = blockDim.x, t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5, nwarps = T >> 5;
    int carry = 0;  // picked blocks in the tiles before this one
    for (int base = 0; base < nb; base += T * W) {
        const int lo = base + t * W;
        // a warp reads its 32 x 32 flags one coalesced row at a time; lane k
        // keeps the ballot of row k, i.e. the flags lo .. lo + 31 of its own
        const int wbase = base + warp * 32 * W;
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int b = wbase + k * 32 + lane;
            const unsigned row = __ballot_sync(FULL, b < nb && pick(b));
            if (lane == k) m = row;
        }
        const int cnt = __popc(m);
        // exclusive prefix of cnt over the CTA
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nwarps ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += v;
            }
            warp_sum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        int r = carry + (warp ? warp_sum[warp - 1] : 0) + incl - cnt;
        carry += warp_sum[nwarps - 1];
        while (m) {
            const int b = lo + __ffs(m) - 1;
            m &= m - 1u;
            emit(b, r);
            ++r;
        }
        __syncthreads();  // warp_sum is rewritten by the next tile
    }
}

// Deterministic compaction of the candidates of a step (one CTA): the
// criterion marks candidates in any order (cand_mark 1, a provisional slot);
// here they are renumbered in ascending block order, slot n_old + rank
// (scan_blocks over the marks).  Block creation then sets the mark to 2
// (meshed).
// Nothing is done when the pool cannot hold the candidates (block creation
// undoes them).  Every thread of the CTA must call.
__device__ __forceinline__ void order_body(const KParams &kp, int step)
{
    Ctrl *ctrl = kp.ctrl;
    const int par = step & 1;
    const int n_old = __ldcg(&ctrl->n_active[par]);
    const int ncand = __ldcg(&ctrl->ncand[par]);
    if (__ldcg(&ctrl->status) || ncand <= 0 || n_old + ncand > kp.capacity) return;
    scan_blocks(
        kp.nbx * kp.nby * kp.nbz, [&](int b) { return kp.cand_mark[b] == 1u; },
        [&](int b, int r) {
            kp.cand_list[r] = b;
            kp.slot_of[b] = n_old + r;
        });
}

// The same renumbering by counting, for the usual few candidates of a step:
// a candidate's rank is the number of candidates with a smaller block id
// (O(ncand^2 / threads), no pass over every block's mark); bursts of more
// than ORDER_BY_COUNT candidates take order_body's scan.  The counts were
// changed by other CTAs' atomics: read through L2.  Every thread of the CTA
// must call.
constexpr int ORDER_BY_COUNT = 1024;
__device__ __forceinline__ void order_candidates(const KParams &kp, int step)
{
    __shared__ int cand[ORDER_BY_COUNT];
    Ctrl *ctrl = kp.ctrl;
    const int par = step & 1;
    const int n_old = __ldcg(&ctrl->n_active[par]);
    const int ncand = __ldcg(&ctrl->ncand[par]);
    if (__ldcg(&ctrl->status) || ncand <= 0 || n_old + ncand > kp.capacity) return;
    if (ncand > ORDER_BY_COUNT) {
        order_body(kp, step);
        return;
    }
    for (int k = threadIdx.x; k < ncand; k += blockDim.x) cand[k] = __ldcg(kp.cand_list + k);
    __syncthreads();
    for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
        const int b = cand[k];
        int r = 0;
        for (int j = 0; j < ncand; ++j) r += cand[j] < b;
        kp.cand_list[r] = b;
        kp.slot_of[b] = n_old + r;
    }
}

// The last CTA of a pass-1 launch renumbers the step's candidates (block
// creation then needs no launch of its own for it).  Every thread calls.
__device__ void order_tail(const KParams &kp, int step)
{
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&kp.ctrl->macro_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) kp.ctrl->macro_done = 0u;
    order_candidates(kp, step);
}

// ---- slot order ---------------------------------------------------------------
// Blocks created by the criterion take the next free slots, so the slot
// order drifts from the spatial order: a block's neighbours are no longer
// processed near it in time and the sectors they share miss L2 (the same
// meshed set runs its passes about 10 % faster per cell in block order than
// in creation order).  Between steps the meshed slots are renumbered in
// block order once the blocks created since the last renumbering reach
// 1/16 of the meshed ones: k_sort_rank decides and ranks the blocks
// (perm[new slot] = old slot, in cand_list, free between steps), k_sort_aux
// moves the solid words, the previous velocities, the 16-bit forms'
// previous densities, the density partials and block_of through the other
// population buffer
// (idle between steps), k_sort_move / k_sort_back then move the populations
// of the next step's read buffer through it, which leaves both buffers
// holding them, and k_sort_tables
// rebuilds the neighbour-slot table.  The launches after k_sort_rank return
// at once when it decided not to move.  No cell's arithmetic changes: the
// results are the same bit for bit.

__global__ void __launch_bounds__(1024) k_sort_rank(KParams kp)
{
    __shared__ int go;
    Ctrl *ctrl = kp.ctrl;
    const int n = ctrl->n_active[ctrl->step & 1];
    if (threadIdx.x == 0) {
        go = ctrl->status == 0 && n > 0 &&
             (ctrl->created - ctrl->sorted_created) * 16ull >= (unsigned long long)n;
        ctrl->sort_go = go;
    }
    __syncthreads();
    if (!go) return;
    // A-A: no idle buffer to move the blocks through; the passes visit the
    // slots in this order instead
    int *perm = kp.aa ? kp.order : kp.cand_list;
    // rank r of the slot order (block order, or strips of block rows)
    auto blk = [&](int r) { return strip_block(r, kp.nbx, kp.nby, kp.nbz, kp.strip); };
    scan_blocks(
        kp.nbx * kp.nby * kp.nbz, [&](int r) { return kp.slot_of[blk(r)] >= 0; },
        [&](int r, int k) { perm[k] = kp.slot_of[blk(r)]; });
    if (kp.aa && threadIdx.x == 0) {
        ctrl->n_sorted = n;
        ctrl->sorted_created = ctrl->created;
        ctrl->sorts += 1ull;
        ctrl->sort_go = 0;
    }
}

// dst[new][k] = src[perm[new]][k] over `words` words per slot, or a plain
// copy when perm is NULL.
template <class T>
__device__ __forceinline__ void sort_copy(const T *src, T *dst, const int *perm, int n, int words)
{
    const size_t total = (size_t)n * words;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int s2 = (int)(e / words), k = (int)(e % words);
        const int s = perm ? perm[s2] : s2;
        dst[(size_t)s2 * words + k] = src[(size_t)s * words + k];
    }
}

template <int ST>
__global__ void __launch_bounds__(THREADS) k_sort_move(KParams kp)
{
    const Ctrl *ctrl = kp.ctrl;
    if (!ctrl->sort_go) return;
    const int par = ctrl->step & 1;
    const typename Store<ST>::T *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
    typename Store<ST>::T *tmp = pops<ST>(kp) + (size_t)(par ^ 1) * kp.buf_stride;
    sort_copy(rd, tmp, kp.cand_list, ctrl->n_active[par], kp.slot_floats);
}

template <int ST>
__global__ void __launch_bounds__(THREADS) k_sort_back(KParams kp)
{
    const Ctrl *ctrl = kp.ctrl;
    if (!ctrl->sort_go) return;
    const int par = ctrl->step & 1;
    typename Store<ST>::T *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
    const typename Store<ST>::T *tmp = pops<ST>(kp) + (size_t)(par ^ 1) * kp.buf_stride;
    sort_copy(tmp, rd, (const int *)nullptr, ctrl->n_active[par], kp.slot_floats);
}

// The per-slot words of the other arrays (solid words, previous velocities,
// 16-bit forms' previous densities as a float4 per cell, density partials,
// block_of) into slot `new` of the other population buffer, packed, or back
// (BACK).  (A partial entry belongs to the half block that receives it, so
// it moves with that slot.)
template <int ST, bool BACK>
__global__ void __launch_bounds__(THREADS) k_sort_aux(KParams kp)
{
    Ctrl *ctrl = kp.ctrl;
    if (!ctrl->sort_go) return;
    const int par = ctrl->step & 1;
    const int n = ctrl->n_active[par];
    uint32_t *tmp = reinterpret_cast<uint32_t *>(pops<ST>(kp) + (size_t)(par ^ 1) * kp.buf_stride);
    uint32_t *uprev = reinterpret_cast<uint32_t *>(kp.uprev);
    uint32_t *macp = reinterpret_cast<uint32_t *>(kp.mac + (size_t)(par ^ 1) * kp.mac_stride);
    const int nup = kp.uprev ? kp.ncomp * 3 * CELLS : 0;
    const int nmac = Store<ST>::DEV ? 4 * CELLS : 0;
    const int npart = kp.part ? 2 * CELLS : 0;
    const int nrecv = kp.recv ? 2 * PARTS * recv_entries(BX, BY, BZ) : 0;
    uint32_t *partw = reinterpret_cast<uint32_t *>(kp.part);
    uint32_t *recvw = reinterpret_cast<uint32_t *>(kp.recv);
    const int words = CELLS + nup + nmac + npart + nrecv + 1;
    const size_t total = (size_t)n * words;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int s2 = (int)(e / words), k = (int)(e % words);
        uint32_t *t = tmp + (size_t)s2 * kp.slot_floats + k;
        uint32_t *a;  // the word in its own array, at the old slot (move) or the new one (back)
        const int s = BACK ? s2 : kp.cand_list[s2];
        if (k < CELLS)
            a = kp.nbits + (size_t)s * CELLS + k;
        else if (k < CELLS + nup)
            a = uprev + (size_t)s * nup + (k - CELLS);
        else if (k < CELLS + nup + nmac)
            a = macp + (size_t)s * nmac + (k - CELLS - nup);
        else if (k < CELLS + nup + nmac + npart)
            a = partw + (size_t)s * npart + (k - CELLS - nup - nmac);
        else if (k < CELLS + nup + nmac + npart + nrecv)
            a = recvw + (size_t)s * nrecv + (k - CELLS - nup - nmac - npart);
        else
            a = reinterpret_cast<uint32_t *>(kp.block_of + s);
        if (BACK) {
            *a = *t;
            if (k == words - 1) kp.slot_of[(int)*t] = s2;
        } else {
            *t = *a;
        }
    }
}

// The neighbour-slot table of the renumbered slots (as warp_nbr), and the
// bookkeeping of the renumbering.  With the fused step, also the distance
// from each slot to its farthest meshed neighbour, as a histogram; the last
// CTA turns it into ctrl->fz_dist, the distance that covers FZ_COVER_PERMIL
// per mille of the slots (the fused step's lag; the rest are deferred).
__global__ void __launch_bounds__(THREADS) k_sort_tables(KParams kp)
{
    __shared__ int last;
    Ctrl *ctrl = kp.ctrl;
    if (!ctrl->sort_go) return;
    const int n = ctrl->n_active[ctrl->step & 1];
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * (THREADS / 32) + (threadIdx.x >> 5); s < n; s += gridDim.x * (THREADS / 32)) {
        int v = SOLIDBLK;
        if (lane == 13) {
            v = s;
        } else if (lane < 27) {
            const int nid = neighbour_of(kp, kp.block_of[s], lane);
            if (nid >= 0) v = kp.slot_of[nid];
        }
        kp.nbr[(size_t)s * NBR_STRIDE + lane] = v;
        if (kp.fz_hist) {
            const int far = __reduce_max_sync(FULL, v);
            if (lane == 0) atomicAdd(&kp.fz_hist[min((far - s) / FZ_BIN, FZ_BINS - 1)], 1);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->sorted_created = ctrl->created;
        ctrl->sorts += 1ull;
    }
    if (!kp.fz_hist) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctrl->fz_hist_ctas, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        const long long need = ((long long)n * FZ_COVER_PERMIL + 999) / 1000;
        long long cum = 0;
        int b = 0;
        for (; b < FZ_BINS - 1; ++b) {
            cum += __ldcg(kp.fz_hist + b);
            if (cum >= need) break;
        }
        ctrl->fz_dist = (b + 1) * FZ_BIN;
        ctrl->fz_hist_ctas = 0u;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < FZ_BINS; b += blockDim.x) kp.fz_hist[b] = 0;
}

// A-A: one cell of a block created in this step.  Its incoming
// populations, as the A-B pull reads them (a meshed neighbour's value
// towards it; the ambient equilibrium from unmeshed blocks, from blocks
// created in this step and behind solid cells), sit for a source cell in a
// meshed block at (source, opp(i)) after either kind of step: after a local
// step that is where the source's post-collision value is; after a
// neighbour step it is the value the source parked there for this block,
// then unmeshed.  A local step reads them from the cell's own slots, so
// they are copied there; in a neighbour step the new block's slots read as
// the ambient equilibrium.  Then the cell's moments (as macro_cell, in pull
// order) into mac.  wn: the block itself and the blocks created in this
// step map to the ambient slot.  All lanes call.
__device__ __forceinline__ void aa_new_cell(const KParams &kp, const WarpNbr &wn, float4 *mac, int slot,
                                            int gid, int c, int lx, int ly, int lz, uint32_t bits,
                                            int local)
{
    const bool nonsolid = !(bits & 1u);
    const bool held = (bits >> HELD_BIT) & 1u;
    float2 in[Q];
    Unroll<0, Q>::run([&]<int I>() {
        const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
        const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
        const uint32_t o = __shfl_sync(FULL, wn.fbase, k) + (uint32_t)(opp(I) * CELLS + lc);
        const bool from_amb = ((bits >> I) & 1u) || held || !nonsolid;
        in[I] = from_amb ? make_float2(kp.famb[0][I], kp.famb[1][I])
                         : make_float2(__ldg(kp.f + o), __ldg(kp.f + o + Q * CELLS));
    });
    float *d = kp.f + (size_t)slot * kp.slot_floats + c;
    float *hc = held ? kp.held_f + (size_t)kp.held_rank[gid] * kp.slot_floats + c : nullptr;
    Moments m;
    auto one = [&]<int I>() {
        d[I * CELLS] = local ? in[I].x : kp.famb[0][I];
        d[(Q + I) * CELLS] = local ? in[I].y : kp.famb[1][I];
        if (hc) {
            hc[I * CELLS] = kp.famb[0][I];
            hc[(Q + I) * CELLS] = kp.famb[1][I];
        }
        m.template add<I>(0, in[I].x);
        m.template add<I>(1, in[I].y);
    };
    one.template operator()<0>();
    Unroll<0, NPAIR>::run([&]<int P>() {
        one.template operator()<pair_rep(P)>();
        one.template operator()<opp(pair_rep(P))>();
    });
    if (nonsolid) mac[(size_t)slot * CELLS + c] = mac_pack(m.rho[0], psi_of(kp, m.rho[0]), m.rho[1]);
}

// Block creation (Sec. 4.2-4.3): the candidates found by k_macro get slots
// after the meshed ones, start from the ambient resting equilibrium in both
// buffers (the paper gives no state for a new sub-domain; the resting
// ambient keeps an untouched region unchanged) and get their streaming and
// moments of this step computed,
// with every block created in this step seen as ambient.  The deviation
// forms write the read buffer only (the collision of this step writes every
// non-solid cell of the other one), against the previous densities of the
// reading cells, and give the block the ambient density as its previous one.
template <int NC, int ST>
__device__ __forceinline__ void activate_body(const KParams &kp, int step)
{
    using S = Store<ST>;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n_old = ctrl->n_active[par];
    const int ncand = ctrl->ncand[par];
    if (!in_range(kp, ncand, (long long)kp.nbx * kp.nby * kp.nbz + 1, 4)) return;
    if (n_old + ncand > kp.capacity) {
        // the pool cannot hold them: undo the slots k_macro handed out, so
        // the state stays that of the last completed step
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncand; k += gridDim.x * blockDim.x) {
            const int gid = kp.cand_list[k];
            kp.slot_of[gid] = AMBIENT;
            kp.cand_mark[gid] = 0u;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctrl->status = LBM_ENOMEM;
            ctrl->fail_step = step;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->n_active[par ^ 1] = n_old + ncand;
        ctrl->ncand[par ^ 1] = 0;
        ctrl->created += (unsigned long long)ncand;
    }
    typename S::T *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
    float4 *mac = kp.mac + (size_t)par * kp.mac_stride;
    float4 *mac_prev = kp.mac + (size_t)(par ^ 1) * kp.mac_stride;
    for (int it = blockIdx.x; it < ncand * PARTS; it += gridDim.x) {
        const int k = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const int slot = n_old + k;
        const int gid = kp.cand_list[k];
        if (!in_range(kp, gid, (long long)kp.nbx * kp.nby * kp.nbz, 5)) continue;
        if (c == 0) {
            kp.block_of[slot] = gid;
            kp.cand_mark[gid] = 2u;  // meshed
        }
        if (c < 32) {
            // the new block's row of the neighbour-slot table, and its slot in
            // the rows of its meshed neighbours (every candidate's slot is
            // already set, so the two writers of an entry agree)
            int s = SOLIDBLK;
            if (c == 13) {
                s = slot;
            } else if (c < 27) {
                const int nid = neighbour_of(kp, gid, c);
                if (nid >= 0) s = kp.slot_of[nid];
                if (s >= 0 && in_range(kp, s, kp.capacity, 6))
                    kp.nbr[(size_t)s * NBR_STRIDE + (26 - c)] = slot;
            }
            kp.nbr[(size_t)slot * NBR_STRIDE + c] = s;
        }
        // the cell's solid word: prepared ahead by the activation proposer
        // (the same value, computed earlier on a side stream), or computed now
        unsigned prepared = 0;
        if (kp.prep) {
            prepared = *(volatile const unsigned *)&kp.prep[gid];
            __threadfence();
        }
        // (prepared is the same for the whole warp: one load of one word)
        uint32_t bits;
        if (prepared) {
            bits = __ldcg(kp.nbits_pre + (size_t)gid * CELLS + c);
        } else {
            const int lane = threadIdx.x & 31;
            const int nid_lane = lane == 13 ? gid : (lane < 27 ? neighbour_of(kp, gid, lane) : -1);
            bits = cell_bits_nbr(kp, gid, nid_lane, c);
        }
        if (c == 0) {
            kp.act_step[gid] = step + 1;
            if (prepared) atomicAdd(&ctrl->prepared_hits, 1ull);
        }
        kp.nbits[(size_t)slot * CELLS + c] = bits;
        const bool live = !(bits & 1u);
        const unsigned fluid = __ballot_sync(FULL, live && !((bits >> HELD_BIT) & 1u));
        if ((threadIdx.x & 31) == 0 && fluid)
            atomicAdd(&ctrl->fluid_active, (unsigned long long)__popc(fluid));
        const WarpNbr wn = warp_nbr(kp, gid, slot, n_old, true);
        const float4 amb = mac_pack(kp.rho_amb[0], kp.psi_amb, kp.rho_amb[1]);
        if constexpr (!S::DEV && NC == 2) {
            if (kp.aa) {  // warp-uniform
                aa_new_cell(kp, wn, mac, slot, gid, c, lx, ly, lz, bits, step & 1);
                continue;
            }
        }
        if constexpr (!S::DEV) {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float *d0 = kp.f + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
                float *d1 = d0 + kp.buf_stride;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    d0[i * CELLS] = kp.famb[a][i];
                    d1[i * CELLS] = kp.famb[a][i];
                }
            }
        } else {
            // blocks created in this step (slots >= n_old) are ambient
            // readers, like the unmeshed ones
            float rdst[2][Q];
            reader_refs<NC>(wn, mac_prev, lx, ly, lz, bits, live, kp.rho_amb, rdst);
            uint32_t *d = rd + (size_t)slot * kp.slot_floats + c;
            Unroll<0, Q>::run([&]<int I>() {
                d[I * CELLS] = live ? S::enc2(__fmaf_rn(-wgt(I), rdst[0][I], kp.famb[0][I]),
                                              NC == 2 ? __fmaf_rn(-wgt(I), rdst[1][I], kp.famb[1][I]) : 0.f)
                                    : 0u;
            });
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                up[0] = up[CELLS] = up[2 * CELLS] = 0.f;
            }
            mac_prev[(size_t)slot * CELLS + c] = live ? amb : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float rho[2], u[2][3];
        macro_cell<NC, ST>(kp, wn, rd, mac, slot, c, lx, ly, lz, bits, live, true, kp.rho_amb, amb, rho, u);
    }
}

template <int NC, int ST>
__global__ void __launch_bounds__(THREADS) k_activate(KParams kp)
{
    activate_body<NC, ST>(kp, kp.ctrl->step);
}

// Forces on a fluid cell (Eqs. 8-9 as read, gravity, adhesion), from the
// mac values of its 18 neighbours.  A solid neighbour lends the centre's own
// values; an unmeshed one the ambient values.  The mac copy in use starts
// at kp.mac + moff (wn.mbase includes moff; addressing from the kernel
// parameter keeps the gather's address registers down).  With REFS the
// neighbours' densities are also returned per direction (rdst, the reading
// cells' references of the deviation forms).  All lanes must call; `live`
// masks the loads.
template <int NC, bool REFS = false>
__device__ __forceinline__ void forces(const KParams &kp, const WarpNbr &wn, uint32_t moff,
                                       int slot, int c, int lx, int ly, int lz, uint32_t bits,
                                       bool live, const float rho[2], float F[2][3],
                                       float rdst[2][Q] = nullptr)
{
    const float psi_c = live ? kp.mac[(size_t)moff + (size_t)slot * CELLS + c].z : 0.f;
    const float r0c = rho[0], r1c = NC == 2 ? rho[1] : 0.f;
    float sp[3] = {0, 0, 0}, sp2[3] = {0, 0, 0}, sr0[3] = {0, 0, 0}, sr1[3] = {0, 0, 0},
          ss[3] = {0, 0, 0};
    Unroll<0, NPAIR>::run([&]<int P>() {
        constexpr int I = pair_rep(P);
        constexpr int J = opp(I);
        float psi_n[2], r0_n[2], r1_n[2], s_n[2];
        Unroll<0, 2>::run([&]<int H>() {
            constexpr int D = H == 0 ? I : J;
            const int tx = lx + cx(D), ty = ly + cy(D), tz = lz + cz(D);
            const int k = nbk(tx, ty, tz), lc = lcell(tx, ty, tz);
            const uint32_t mb = __shfl_sync(FULL, wn.mbase, k);
            const bool solid_n = (bits >> opp(D)) & 1u;  // x + e_D = x - e_opp(D)
            const float4 m = live ? __ldg(kp.mac + mb + lc) : make_float4(0.f, 0.f, 0.f, 0.f);
            psi_n[H] = solid_n ? psi_c : m.z;
            r0_n[H] = solid_n ? r0c : m.x;
            r1_n[H] = solid_n ? r1c : m.y;
            s_n[H] = solid_n ? 1.f : 0.f;
            if constexpr (REFS) {
                rdst[0][D] = r0_n[H];
                if (NC == 2) rdst[1][D] = r1_n[H];
            }
        });
        const float w = wgt(I);
        const float dp = w * (psi_n[0] - psi_n[1]);
        const float dp2 = w * (psi_n[0] * psi_n[0] - psi_n[1] * psi_n[1]);
        const float d0 = w * (r0_n[0] - r0_n[1]);
        const float d1 = w * (r1_n[0] - r1_n[1]);
        const float ds = w * (s_n[0] - s_n[1]);
        const int e[3] = {cx(I), cy(I), cz(I)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (e[d] > 0) {
                sp[d] += dp; sp2[d] += dp2; sr0[d] += d0; sr1[d] += d1; ss[d] += ds;
            } else if (e[d] < 0) {
                sp[d] -= dp; sp2[d] -= dp2; sr0[d] -= d0; sr1[d] -= d1; ss[d] -= ds;
            }
        }
    });
    const float a1 = -kp.beta * kp.g_self * psi_c;
    const float a2 = -(1.f - kp.beta) * 0.5f * kp.g_self;
    const float ex0 = fmaxf(r0c - kp.rho_amb[0], 0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float f0 = a1 * sp[d] + a2 * sp2[d] - kp.g_ads[0] * ex0 * ss[d] +
                   (r0c - kp.rho_ref[0]) * kp.grav[d];
        if (NC == 2) f0 -= kp.g_cross * r0c * sr1[d];
        F[0][d] = f0;
    }
    if (NC == 2) {
        const float ex1 = fmaxf(r1c - kp.rho_amb[1], 0.f);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            F[1][d] = -kp.g_cross * r1c * sr0[d] - kp.g_ads[1] * ex1 * ss[d] +
                      (r1c - kp.rho_ref[1]) * kp.grav[d];
    }
}

// Pass 2 of a step (FP32 form): streaming again, forces, forced BGK
// collision (Eqs. 10-12, read with the stable sign -(f - f_eq) / tau of
// standard BGK), store into the other buffer; the
// velocity is kept for the next criterion at cells that border unmeshed
// blocks.
template <int NC, bool TAU1>
__device__ __forceinline__ void collide_body(const KParams &kp, int step)
{
    constexpr int ST = LBM_STORAGE_FP32;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 7)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    float *wr = kp.f + (size_t)(par ^ 1) * kp.buf_stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    const int total = n * PARTS;
    int it = blockIdx.x;
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, next_row);
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        const bool live = !(bits & 1u) && !((bits >> HELD_BIT) & 1u);
        // every lane takes part in the ballot (it must not sit behind &&)
        const bool row_live = row_has(live);
        const bool fill = (bits & 1u) && row_live;  // solid cell completing a sector
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 8))) continue;
        Moments m;
        float fin[TAU1 ? 1 : NC][Q];
        const float ref[2] = {0.f, 0.f};
        pull<NC, ST>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false, ref,
                     [&]<int I>(int a, float v) {
                         m.template add<I>(a, v);
                         if constexpr (!TAU1) fin[a][I] = v;
                     });
        float rho[2] = {m.rho[0], m.rho[1]}, u[2][3];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const float inv = 1.f / rho[a];
            u[a][0] = m.j[a][0] * inv;
            u[a][1] = m.j[a][1] * inv;
            u[a][2] = m.j[a][2] * inv;
        }
        float F[2][3];
        forces<NC>(kp, wn, 0u, slot, c, lx, ly, lz, bits, live, rho, F);
        if (!live && !fill) continue;
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            const float inv = 1.f / rho[a];
            const float vx = u[a][0] + F[a][0] * inv, vy = u[a][1] + F[a][1] * inv,
                        vz = u[a][2] + F[a][2] * inv;
            const float vv = vx * vx + vy * vy + vz * vz;
            const float uu = u[a][0] * u[a][0] + u[a][1] * u[a][1] + u[a][2] * u[a][2];
            float *dst = wr + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
            const float r = rho[a];
            // The 18 moving populations from Eqs. 10-12; the rest population
            // from the mass balance sum_i f_i = rho, which the collision
            // satisfies exactly in real arithmetic.  In FP32 this keeps the
            // mass free of the systematic bias of the rounded weights
            // (fl(1/3) + 6 fl(1/18) + 12 fl(1/36) = 1 + 1.5e-8).
            float moving = 0.f;
            Unroll<1, Q>::run([&]<int I>() {
                const float wr_ = wgt(I) * r;
                float v = feq<I>(wr_, vx, vy, vz, vv);
                if constexpr (!TAU1) {
                    const float e0 = feq<I>(wr_, u[a][0], u[a][1], u[a][2], uu);
                    v += (1.f - kp.omega) * (fin[a][I] - e0);
                }
                moving += v;
                dst[I * CELLS] = live ? v : 0.f;
            });
            dst[0] = live ? r - moving : 0.f;
        }
        if (live && kp.progressive && (reach_bits(lx, ly, lz) & wn.amb)) {
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                up[0] = u[a][0];
                up[CELLS] = u[a][1];
                up[2 * CELLS] = u[a][2];
            }
        }
    }
}

template <int NC, bool TAU1>
__global__ void __launch_bounds__(THREADS) k_collide(KParams kp)
{
    const int step = *(volatile const int *)&kp.ctrl->step;
    collide_body<NC, TAU1>(kp, step);
    step_done(kp.ctrl, step);
}

// forces() for both components at once (same terms, paired arithmetic):
// F[d] = (F_0, F_1) along axis d.  The mac copy in use starts at kp.mac +
// moff.  All lanes must call; `live` masks the loads.
// rn (optional): rn[D * THREADS] receives the density pair used for the
// neighbour x + e_D (the cell's own behind a solid neighbour), for the
// 16-bit collision's encode.
template <int NC>
__device__ __forceinline__ void forces2(const KParams &kp, const WarpNbr &wn, uint32_t moff, int slot,
                                        int c, int lx, int ly, int lz, uint32_t bits, bool live,
                                        float2 rho, float2 F[3], float2 *rn = nullptr)
{
    const float psi_c = live ? kp.mac[(size_t)moff + (size_t)slot * CELLS + c].z : 0.f;
    const float2 pc = make_float2(psi_c, psi_c * psi_c);
    float2 sr[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // (sum w rho0 e, sum w rho1 e)
    float2 sp[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};  // (sum w psi e, sum w psi^2 e)
    float ss[3] = {0.f, 0.f, 0.f};                        // sum w s e
    Unroll<0, NPAIR>::run([&]<int P>() {
        constexpr int I = pair_rep(P);
        constexpr int J = opp(I);
        float2 r_n[2], p_n[2];
        float s_n[2];
        Unroll<0, 2>::run([&]<int H>() {
            constexpr int D = H == 0 ? I : J;
            const int tx = lx + cx(D), ty = ly + cy(D), tz = lz + cz(D);
            const int k = nbk(tx, ty, tz), lc = lcell(tx, ty, tz);
            const uint32_t mb = __shfl_sync(FULL, wn.mbase, k);
            const bool solid_n = (bits >> opp(D)) & 1u;  // x + e_D = x - e_opp(D)
            const float4 m = live ? __ldg(kp.mac + mb + lc) : make_float4(0.f, 0.f, 0.f, 0.f);
            r_n[H] = sel2(solid_n, rho, make_float2(m.x, m.y));
            if (rn) rn[D * THREADS] = r_n[H];
            p_n[H] = sel2(solid_n, pc, make_float2(m.z, m.z * m.z));
            s_n[H] = solid_n ? 1.f : 0.f;
        });
        const float2 w = splat(wgt(I));
        const float2 dr = mul2(w, sub2(r_n[0], r_n[1]));
        const float2 dp = mul2(w, sub2(p_n[0], p_n[1]));
        const float ds = wgt(I) * (s_n[0] - s_n[1]);
        const int e[3] = {cx(I), cy(I), cz(I)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (e[d] > 0) {
                sr[d] = add2(sr[d], dr); sp[d] = add2(sp[d], dp); ss[d] += ds;
            } else if (e[d] < 0) {
                sr[d] = sub2(sr[d], dr); sp[d] = sub2(sp[d], dp); ss[d] -= ds;
            }
        }
    });
    // cohesion (component 0), cross force, adhesion, gravity
    const float a1 = -kp.beta * kp.g_self * psi_c;
    const float a2 = -(1.f - kp.beta) * 0.5f * kp.g_self;
    const float2 cross = NC == 2 ? make_float2(-kp.g_cross * rho.x, -kp.g_cross * rho.y)
                                 : make_float2(0.f, 0.f);
    const float2 ads = make_float2(-kp.g_ads[0] * fmaxf(rho.x - kp.rho_amb[0], 0.f),
                                   NC == 2 ? -kp.g_ads[1] * fmaxf(rho.y - kp.rho_amb[1], 0.f) : 0.f);
    const float2 buoy = make_float2(rho.x - kp.rho_ref[0], NC == 2 ? rho.y - kp.rho_ref[1] : 0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float2 coh = make_float2(a1 * sp[d].x + a2 * sp[d].y, 0.f);
        const float2 swapped = make_float2(sr[d].y, sr[d].x);  // the other component's sum
        F[d] = fma2(cross, swapped, fma2(ads, splat(ss[d]), fma2(buoy, splat(kp.grav[d]), coh)));
    }
}

// Shared by the paired collision kernels: e . a for a velocity vector a
// given with its negation na (no arithmetic for a single nonzero
// component).
template <int I>
__device__ __forceinline__ float2 edot(const float2 *a, const float2 *na)
{
    float2 r = make_float2(0.f, 0.f);
    bool any = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int e = d == 0 ? cx(I) : (d == 1 ? cy(I) : cz(I));
        if (e == 0) continue;
        const float2 t = e > 0 ? a[d] : na[d];
        r = any ? add2(r, t) : t;
        any = true;
    }
    return r;
}

// ---- density partials (FP32, two components, A-B) ----------------------------
// Pull streaming (Eq. 10, left) makes the density of cell y at step t + 1 the
// sum of the post-collision values f*_i(y - e_i) of step t (the cell's own
// f*_opp(i) behind a solid cell, its own stored values at held cells), so
// the collision of step t already holds every term of it.  Each CTA, once
// its half block is collided, sums in shared memory
//   own partial  for each of its cells, the terms that come from the half
//                block itself (part, one float2 per cell);
//   entries      for each cell just outside it, the terms it sends there,
//                stored with the receiving half block (recv).
// Pass 1 of step t + 1 then adds a cell's own partial and the entries of its
// faces and edges (Eqs. 4, 6, 7) instead of pulling 38 populations, wherever
// the warp's 27 blocks are all meshed (or solid); elsewhere, where the
// criterion needs the velocity too, it pulls as before.  The sums are taken
// in a fixed order, so every execution mode gives the same bits; they differ
// from the pull's running sum only by rounding order.
//
// The entries of a half block (HX x HY x HZ cells; blocks split in two along
// z) are grouped by the side they come from: region R has the offset
// (dx, dy, dz) of the sending half block, faces 0-5 (-x, +x, -y, +y, -z, +z)
// then the 12 edges; within a region, the receiving cells in x, y, z order
// over the axes where the offset is 0.
constexpr int HX = BX, HY = BY, HZ = BZ / PARTS;
constexpr int NREG = 18;
// dynamic shared memory of a collision that writes the partials: two
// buffers of the 19 value pairs of a half block's cells
constexpr size_t PART_SMEM = 2 * (size_t)Q * THREADS * sizeof(float2);
static_assert(PARTS == 2, "half blocks along z");
__host__ __device__ constexpr int reg_dx(int r)
{
    return (r == 0 || r == 6 || r == 8 || r == 10 || r == 12) ? -1
           : (r == 1 || r == 7 || r == 9 || r == 11 || r == 13) ? 1
                                                                 : 0;
}
__host__ __device__ constexpr int reg_dy(int r)
{
    return (r == 2 || r == 6 || r == 7 || r == 14 || r == 16) ? -1
           : (r == 3 || r == 8 || r == 9 || r == 15 || r == 17) ? 1
                                                                 : 0;
}
__host__ __device__ constexpr int reg_dz(int r)
{
    return (r == 4 || r == 10 || r == 11 || r == 14 || r == 15) ? -1
           : (r == 5 || r == 12 || r == 13 || r == 16 || r == 17) ? 1
                                                                   : 0;
}
__host__ __device__ constexpr int reg_size(int r)
{
    return (reg_dx(r) == 0 ? HX : 1) * (reg_dy(r) == 0 ? HY : 1) * (reg_dz(r) == 0 ? HZ : 1);
}
__host__ __device__ constexpr int reg_base(int r) { return r == 0 ? 0 : reg_base(r - 1) + reg_size(r - 1); }
constexpr int RECV = reg_base(NREG);
static_assert(RECV == recv_entries(BX, BY, BZ), "entries per half block");

// Position of a receiving cell (x, y, z; half-block coordinates) in region R.
template <int R>
__device__ __forceinline__ int reg_pos(int x, int y, int z)
{
    int p = 0, m = 1;
    if constexpr (reg_dx(R) == 0) { p += x * m; m *= HX; }
    if constexpr (reg_dy(R) == 0) { p += y * m; m *= HY; }
    if constexpr (reg_dz(R) == 0) p += z * m;
    return p;
}
// Whether cell (x, y, z) of a half block borders region R.
template <int R>
__device__ __forceinline__ bool reg_touch(int x, int y, int z)
{
    return (reg_dx(R) == 0 || x == (reg_dx(R) < 0 ? 0 : HX - 1)) &&
           (reg_dy(R) == 0 || y == (reg_dy(R) < 0 ? 0 : HY - 1)) &&
           (reg_dz(R) == 0 || z == (reg_dz(R) < 0 ? 0 : HZ - 1));
}
// Neighbour-block index (0..26) of the half block at offset (ox, oy, oz),
// in half blocks, from half h of a block, and that half block's half.
__device__ __forceinline__ int half_nbr(int ox, int oy, int oz, int h, int &hn)
{
    int zh = h + oz, bz = 0;
    if (zh < 0) {
        zh += PARTS;
        bz = -1;
    } else if (zh >= PARTS) {
        zh -= PARTS;
        bz = 1;
    }
    hn = zh;
    return (ox + 1) + 3 * (oy + 1) + 9 * (bz + 1);
}

// After the collision of half block h of `slot` put every cell's values in
// sv[i][cell] (post-collision values; zeros at solid cells; the stored
// values at held cells): this cell's own partial, then the entries this half
// block sends (a warp-uniform loop; receivers that are unmeshed or solid
// get none).  All threads of the CTA call, between two barriers.
__device__ __forceinline__ void part_write(const KParams &kp, const float2 (*sv)[THREADS], int slot,
                                           int h, int c, uint32_t bits)
{
    const int cl = c - h * THREADS;
    const int lx = lx_of(c), ly = ly_of(c), hz = lz_of(c) - h * HZ;
    const bool held = (bits >> HELD_BIT) & 1u;
    const float2 *me = &sv[0][cl];  // sv[i][cl - d] == me[i * THREADS - d]
    float2 s = me[0];
    auto one = [&]<int I>() {
        constexpr int D = cx(I) + HX * (cy(I) + HY * cz(I));  // cell offset of x - e_I
        const bool inside = (cx(I) == 0 || (cx(I) > 0 ? lx > 0 : lx < HX - 1)) &&
                            (cy(I) == 0 || (cy(I) > 0 ? ly > 0 : ly < HY - 1)) &&
                            (cz(I) == 0 || (cz(I) > 0 ? hz > 0 : hz < HZ - 1));
        if (held)
            s = add2(s, me[I * THREADS]);
        else if ((bits >> I) & 1u)
            s = add2(s, me[opp(I) * THREADS]);
        else if (inside)
            s = add2(s, me[I * THREADS - D]);
    };
    Unroll<0, NPAIR>::run([&]<int P>() {
        one.template operator()<pair_rep(P)>();
        one.template operator()<opp(pair_rep(P))>();
    });
    kp.part[(size_t)slot * CELLS + c] = (bits & 1u) ? make_float2(0.f, 0.f) : s;
    const int *row = kp.nbr + (size_t)slot * NBR_STRIDE;
    for (int e = threadIdx.x; e < RECV; e += THREADS) {
        Unroll<0, NREG>::run([&]<int R>() {
            constexpr int DX = reg_dx(R), DY = reg_dy(R), DZ = reg_dz(R);
            if (e < reg_base(R) || e >= reg_base(R) + reg_size(R)) return;
            // the receiving cell, in the receiver's coordinates
            int p = e - reg_base(R);
            int x = DX < 0 ? 0 : HX - 1, y = DY < 0 ? 0 : HY - 1, z = DZ < 0 ? 0 : HZ - 1;
            if constexpr (DX == 0) { x = p % HX; p /= HX; }
            if constexpr (DY == 0) { y = p % HY; p /= HY; }
            if constexpr (DZ == 0) z = p;
            // its sources x - e_i that lie in this half block (at offset
            // (DX, DY, DZ) from the receiver), in pull order
            float2 sum = make_float2(0.f, 0.f);
            Unroll<0, NPAIR>::run([&]<int P>() {
                Unroll<0, 2>::run([&]<int K>() {
                    constexpr int I = K == 0 ? pair_rep(P) : opp(pair_rep(P));
                    if constexpr ((DX == 0 || cx(I) == -DX) && (DY == 0 || cy(I) == -DY) &&
                                  (DZ == 0 || cz(I) == -DZ)) {
                        const int sx = x - cx(I) - DX * HX, sy = y - cy(I) - DY * HY, sz = z - cz(I) - DZ * HZ;
                        if (sx >= 0 && sx < HX && sy >= 0 && sy < HY && sz >= 0 && sz < HZ)
                            sum = add2(sum, sv[I][sx + HX * (sy + HY * sz)]);
                    }
                });
            });
            int hn;
            const int k = half_nbr(-DX, -DY, -DZ, h, hn);
            const int rs = row[k];
            if (rs >= 0) kp.recv[((size_t)rs * PARTS + hn) * RECV + e] = sum;
        });
    }
}

// Pass 1 from the partials: the density pair of cell c (not solid, not
// held) of half block h, from its own partial `own` and the entries of the
// regions it borders whose sending block exists (bit k of `exist`: block k
// of the 27 is meshed; unmeshed ones do not occur here, solid ones send
// nothing because every source in them is solid).
__device__ __forceinline__ float2 part_gather(const KParams &kp, unsigned exist, int slot, int h, int c,
                                              float2 own)
{
    const int lx = lx_of(c), ly = ly_of(c), hz = lz_of(c) - h * HZ;
    const float2 *in = kp.recv + ((size_t)slot * PARTS + h) * RECV;
    float2 rho = own;
    Unroll<0, NREG>::run([&]<int R>() {
        int hn;
        const int k = half_nbr(reg_dx(R), reg_dy(R), reg_dz(R), h, hn);
        if (reg_touch<R>(lx, ly, hz) && ((exist >> k) & 1u))
            rho = add2(rho, in[reg_base(R) + reg_pos<R>(lx, ly, hz)]);
    });
    return rho;
}

// Pass 1 of one cell from the partials: mac (densities and psi, Eqs. 4, 6,
// 7) from the own partial and, for cells neither solid nor held, the
// entries (held cells pull only their own values).  row: this lane's entry
// of the slot's neighbour row; every lane of the warp calls.
__device__ __forceinline__ void part_mac(const KParams &kp, int slot, int c, int row, uint32_t bits, float2 own)
{
    const unsigned exist = __ballot_sync(FULL, row >= 0);
    const bool live = !(bits & 1u);
    float2 rho = own;
    if (live && !((bits >> HELD_BIT) & 1u)) rho = part_gather(kp, exist, slot, c / THREADS, c, rho);
    kp.mac[(size_t)slot * CELLS + c] =
        live ? mac_pack(rho.x, psi_of(kp, rho.x), rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// One work item of pass 1, FP32 form with two components, paired
// arithmetic (as k_macro): streaming and moments of the cells c of one half
// block (row: the slot's neighbour-table entry of this lane, bits: the
// cell's solid word); with `criterion`, Eq. 13 at cells bordering unmeshed
// blocks.  par, n: the step's parity and meshed count.  CG: the populations
// and previous velocities were written earlier in the same launch.
// part_in: the densities come from the partials the previous collision
// wrote, in warps whose 27 blocks are all meshed or solid (own_part: the
// cell's own partial, loaded ahead by the caller).  All lanes of the warp
// call.
// Called by the item functions once the pull's loads are consumed (the
// fused step publishes the previous item's completion there).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

template <bool CG, class Hook = NoHook>
__device__ __forceinline__ void macro2_item(const KParams &kp, Ctrl *ctrl, const float *rd, int par, int n,
                                            int slot, int c, int row, uint32_t bits, int criterion,
                                            bool part_in = false, float2 own_part = float2{},
                                            Hook &&hook = Hook{})
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    const WarpNbr wn = warp_nbr_of(kp, row);
    const bool live = !(bits & 1u);
    const bool held = (bits >> HELD_BIT) & 1u;
    if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 2))) {
        hook();
        return;
    }
    if (part_in && wn.amb == 0u) {  // warp-uniform
        hook();
        part_mac(kp, slot, c, row, bits, own_part);
        return;
    }
    if (!criterion || wn.amb == 0u) {
        // warp-uniform: no cell of the warp borders an unmeshed block, so
        // the criterion has nothing to test and only the densities are
        // needed (summed in the same order as Moments2)
        float2 rho = make_float2(0.f, 0.f);
        pull2_f32<CG>(kp, wn, rd, slot, c, lx, ly, lz, bits, live,
                      [&]<int I>(float2 v) { rho = add2(rho, v); });
        hook();
        kp.mac[(size_t)slot * CELLS + c] =
            live ? mac_pack(rho.x, psi_of(kp, rho.x), rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    Moments2 m;
    pull2_f32<CG>(kp, wn, rd, slot, c, lx, ly, lz, bits, live,
                  [&]<int I>(float2 v) { m.template add<I>(v); });
    hook();
    const float2 inv = make_float2(1.f / m.rho.x, 1.f / m.rho.y);
    float u[2][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float2 ud = mul2(m.j[d], inv);
        u[0][d] = ud.x;
        u[1][d] = ud.y;
    }
    // solid cells write zeros too (never read): complete sectors
    kp.mac[(size_t)slot * CELLS + c] =
        live ? mac_pack(m.rho.x, psi_of(kp, m.rho.x), m.rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
    criterion_mark<2, CG>(kp, ctrl, par, n, slot, c, wn, live && !held, u);
}

// Pass 1 of a step, FP32 form with two components (grid-stride over the
// half-block items of the meshed slots).
__device__ __forceinline__ void macro2_body(const KParams &kp, int step, int criterion, bool part_in)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    const int total = n * PARTS;
    int it = blockIdx.x;
    // the next item's table row, solid word and (with the partials) own
    // partial are loaded one item ahead
    auto cell_of = [&](int i) { return (size_t)(i / PARTS) * CELLS + (i % PARTS) * THREADS + threadIdx.x; };
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits = it < total ? kp.nbits[cell_of(it)] : 1u;
    float2 next_part = part_in && it < total ? kp.part[cell_of(it)] : make_float2(0.f, 0.f);
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int row = next_row;
        const uint32_t bits = next_bits;
        const float2 own_part = next_part;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[cell_of(it2)];
            if (part_in) next_part = kp.part[cell_of(it2)];
        }
        macro2_item<false>(kp, ctrl, rd, par, n, slot, c, row, bits, criterion, part_in, own_part);
    }
}

__global__ void __launch_bounds__(THREADS, 3) k_macro2(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    macro2_body(kp, step, criterion, kp.part_in != 0);
    if (criterion) order_tail(kp, step);
}

// Pass 1 split in two launches when the partials are there (FP32, two
// components, A-B).  k_macro2p: the warps whose 27 blocks are all meshed or
// solid, from the partials; a light kernel (few registers, many warps in
// flight, the next item's table row loaded ahead).  k_macro2f: the other
// warps (they border an unmeshed block, so only a progressive mesh has
// them), pulled as in k_macro2 with the criterion; its last CTA renumbers
// the candidates.  Together they write what one k_macro2 launch with
// kp.part_in writes, bit for bit.
__global__ void __launch_bounds__(THREADS, 6) k_macro2p(KParams kp)
{
    const Ctrl *ctrl = kp.ctrl;
    const int par = ctrl->step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const int total = n * PARTS;
    int it = blockIdx.x;
    int row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int it2 = it + gridDim.x;
        const int next_row = it2 < total ? nbr_row_lane(kp, it2 / PARTS) : SOLIDBLK;
        const unsigned amb = __ballot_sync(FULL, row == AMBIENT) & ~(1u << 13);
        const bool ok = __all_sync(FULL, in_range(kp, row + 2, (long long)kp.capacity + 2, 2));
        if (amb == 0u && ok) {
            const size_t cell = (size_t)slot * CELLS + c;
            part_mac(kp, slot, c, row, kp.nbits[cell], kp.part[cell]);
        }
        row = next_row;
    }
}

__device__ __forceinline__ void macro2_frontier_body(const KParams &kp, int step, int criterion)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    const int total = n * PARTS;
    int it = blockIdx.x;
    int row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int it2 = it + gridDim.x;
        const int next_row = it2 < total ? nbr_row_lane(kp, it2 / PARTS) : SOLIDBLK;
        if (__ballot_sync(FULL, row == AMBIENT) & ~(1u << 13))  // warp-uniform
            macro2_item<false>(kp, ctrl, rd, par, n, slot, c, row, kp.nbits[(size_t)slot * CELLS + c],
                               criterion);
        row = next_row;
    }
}

__global__ void __launch_bounds__(THREADS, 3) k_macro2f(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    macro2_frontier_body(kp, step, criterion);
    if (criterion) order_tail(kp, step);
}

// One work item of pass 2, FP32 form with two components, paired
// arithmetic (as k_collide): streaming again, forces from the neighbours'
// mac, forced BGK collision into the write buffer, the velocity kept at
// cells bordering unmeshed blocks.  PART: also every cell's values in
// sv[i][cell of the half block] for the density partials.  All lanes of the
// warp call.
template <bool TAU1, bool PART = false, class Hook = NoHook, class Mid = NoMid>
__device__ __forceinline__ void collide2_item(const KParams &kp, const float *rd, float *wr, int slot, int c,
                                              int row, uint32_t bits, float2 (*sv)[THREADS] = nullptr,
                                              Hook &&hook = Hook{}, Mid &&mid = Mid{})
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    const WarpNbr wn = warp_nbr_of(kp, row);
    const bool held = (bits >> HELD_BIT) & 1u;
    const bool live = !(bits & 1u) && !held;
    const int cl = c & (THREADS - 1);
    // every lane takes part in the ballot (it must not sit behind &&)
    const bool row_live = row_has(live);
    const bool fill = (bits & 1u) && row_live;  // solid cell completing a sector
    if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 8))) {
        hook();
        mid();
        return;
    }
    Moments2 m;
    float2 fin[TAU1 ? 1 : Q];
    pull2_f32(
        kp, wn, rd, slot, c, lx, ly, lz, bits, live,
        [&]<int I>(float2 v) {
            m.template add<I>(v);
            if constexpr (!TAU1) fin[I] = v;
        },
        mid);
    hook();
    const float2 rho = m.rho;
    const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
    float2 u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = mul2(m.j[d], inv);
    float2 F[3];
    forces2<2>(kp, wn, 0u, slot, c, lx, ly, lz, bits, live, rho, F);
    if constexpr (PART) {
        if (held) {  // its stored values, which its neighbours pull
            const float *own = rd + (size_t)slot * kp.slot_floats + c;
#pragma unroll
            for (int i = 0; i < Q; ++i) sv[i][cl] = make_float2(own[i * CELLS], own[(Q + i) * CELLS]);
        } else if (!live && !fill) {
#pragma unroll
            for (int i = 0; i < Q; ++i) sv[i][cl] = make_float2(0.f, 0.f);
        }
    }
    if (!live && !fill) return;
    float2 v[3], nv[3], nu[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        v[d] = fma2(F[d], inv, u[d]);
        nv[d] = sub2(make_float2(0.f, 0.f), v[d]);
        nu[d] = sub2(make_float2(0.f, 0.f), u[d]);
    }
    const float2 one = splat(1.f);
    const float2 cv = fma2(splat(-1.5f), fma2(v[0], v[0], fma2(v[1], v[1], mul2(v[2], v[2]))), one);
    const float2 cu = fma2(splat(-1.5f), fma2(u[0], u[0], fma2(u[1], u[1], mul2(u[2], u[2]))), one);
    float2 wrho[3];
    Unroll<0, 3>::run([&]<int K>() {
        constexpr int I = K == 0 ? 0 : (K == 1 ? 1 : 5);
        wrho[K] = mul2(splat(wgt(I)), rho);
    });
    const float2 relax = splat(1.f - kp.omega);
    float2 moving = make_float2(0.f, 0.f);
    float *d0 = wr + (size_t)slot * kp.slot_floats + c;
    float *d1 = d0 + Q * CELLS;
    // the 18 moving populations (Eqs. 10-12); the rest population from
    // the mass balance sum_i f_i = rho (see k_collide)
    Unroll<1, Q>::run([&]<int I>() {
        const float2 ev = edot<I>(v, nv);
        float2 f = mul2(wrho[wclass(I)], fma2(ev, fma2(ev, splat(4.5f), splat(3.f)), cv));
        if constexpr (!TAU1) {
            const float2 eu = edot<I>(u, nu);
            const float2 e0 = mul2(wrho[wclass(I)], fma2(eu, fma2(eu, splat(4.5f), splat(3.f)), cu));
            f = fma2(relax, sub2(fin[I], e0), f);
        }
        moving = add2(moving, f);
        d0[I * CELLS] = live ? f.x : 0.f;
        d1[I * CELLS] = live ? f.y : 0.f;
        if constexpr (PART) sv[I][cl] = live ? f : make_float2(0.f, 0.f);
    });
    const float2 rest = sub2(rho, moving);
    d0[0] = live ? rest.x : 0.f;
    d1[0] = live ? rest.y : 0.f;
    if constexpr (PART) sv[0][cl] = live ? rest : make_float2(0.f, 0.f);
    (void)cu;
    if (live && kp.progressive && (reach_bits(lx, ly, lz) & wn.amb)) {
        float *up = kp.uprev + (size_t)slot * 2 * 3 * CELLS + c;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            up[d * CELLS] = u[d].x;
            up[(3 + d) * CELLS] = u[d].y;
        }
    }
}

// Pass 2 of a step, FP32 form with two components (grid-stride over the
// half-block items); PART: with the density partials of the next step (the
// launch then gives PART_SMEM bytes of dynamic shared memory).
template <bool TAU1, bool PART = false>
__device__ __forceinline__ void collide2_body(const KParams &kp, int step)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int buf = 0, prev_slot = -1, prev_h = 0;
    uint32_t prev_bits = 0;
    (void)buf;
    (void)prev_h;
    (void)prev_bits;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 7)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    float *wr = kp.f + (size_t)(par ^ 1) * kp.buf_stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    const int total = n * PARTS;
    int it = blockIdx.x;
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int row = next_row;
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        if constexpr (PART) {
            // Two buffers of PART_SMEM / 2 bytes, alternating by item.  The
            // partial sums of an item run in the next item's collision,
            // after its loads are issued (their latency hides them), past
            // a barrier that every warp reaches only once it has written
            // the item's values and finished the sums of the item before,
            // which used the buffer this item writes.
            float2 (*base)[THREADS] = reinterpret_cast<float2 (*)[THREADS]>(smem_raw);
            float2 (*sv)[THREADS] = base + (size_t)buf * Q;
            float2 (*pv)[THREADS] = base + (size_t)(buf ^ 1) * Q;
            auto mid = [&]() {
                __syncthreads();
                if (prev_slot >= 0) part_write(kp, pv, prev_slot, prev_h, prev_h * THREADS + threadIdx.x, prev_bits);
            };
            collide2_item<TAU1, true>(kp, rd, wr, slot, c, row, bits, sv, NoHook{}, mid);
            prev_slot = slot;
            prev_h = it % PARTS;
            prev_bits = bits;
            buf ^= 1;
        } else {
            collide2_item<TAU1>(kp, rd, wr, slot, c, row, bits);
        }
    }
    if constexpr (PART) {  // the sums of the last item
        __syncthreads();
        if (prev_slot >= 0)
            part_write(kp, reinterpret_cast<float2 (*)[THREADS]>(smem_raw) + (size_t)(buf ^ 1) * Q, prev_slot,
                       prev_h, prev_h * THREADS + threadIdx.x, prev_bits);
    }
}

template <bool TAU1, bool PART>
__global__ void __launch_bounds__(THREADS, 2) k_collide2(KParams kp)
{
    const int step = *(volatile const int *)&kp.ctrl->step;
    collide2_body<TAU1, PART>(kp, step);
    step_done(kp.ctrl, step);
}

// ---- fused step: the collision of step t and pass 1 of step t + 1 -----------
// (FP32, two components, A-B.)  One launch runs both passes over the meshed
// slots, so that pass 1 reads the populations the collision has just written
// while they are still in L2, instead of from HBM in a launch of its own:
// every population crosses HBM once per step in each direction.
//
// Pass 1 of a half block reads the new populations of its block and of its
// 26 neighbours, and rewrites its block's mac, which the neighbours'
// collisions read.  So it starts only once the collisions of all 27 blocks
// have finished: every warp of a collision item adds 1 to the item's
// counter (release) after its own stores, and pass 1 waits until the
// counters of its neighbourhood read WARPS_PER_ITEM (acquire), then reads
// the populations and previous velocities through L2 (ld.global.cg).  The
// counters come in two parities by step: a launch counts in one and clears
// the other for the next launch (the host clears both after an unfused step).
//
// The work is a fixed sequence: the first L collision items, then collision
// and pass-1 items alternately, then the remaining pass-1 items; CTA g takes
// positions g, g + G, ... in order, its warps each their own rows of every
// item, with no CTA barrier.  The lag L is about the slot distance of a
// block's farthest neighbour (ctrl->fz_dist, see k_sort_tables) plus one
// round of the grid, so that the collisions a pass-1 item needs are a round
// or more behind it.  A pass-1 item waits only for collisions placed before
// it; one whose neighbourhood holds a collision placed after it (a block
// meshed since the last renumbering, a neighbour across a periodic boundary
// or a strip border) is skipped and redone once the CTA's sequence is
// through.  Waits thus only ever point back in the sequence, and every
// wait is bounded anyway (LBM_ETIMEOUT).  The results equal those of
// k_collide2 + k_macro2 bit for bit: the same item code computes every value.

// A strong (L2) load without acquire semantics: polling with acquire loads
// would invalidate the SM's L1 at every poll, under the other warps'
// cached data.  The polled counters are released by their writers; the data
// they guard is then read through L2 (ld.global.cg), so no stale L1 line
// can be seen.
__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Positions in the work sequence of C collision and C pass-1 items with lag
// L (0 <= L <= C), and the item at a position q < 2C.
__device__ __forceinline__ int fz_pos_collide(int i, int L) { return i < L ? i : 2 * i - L; }
enum FzKind { FZ_COLLIDE = 0, FZ_PASS1 = 1 };
__device__ __forceinline__ int fz_item(int q, int C, int L, int &idx)
{
    if (q < L) {
        idx = q;
        return FZ_COLLIDE;
    }
    if (q < 2 * C - L) {
        const int r = (q - L) >> 1;
        idx = ((q - L) & 1) ? r : L + r;
        return ((q - L) & 1) ? FZ_PASS1 : FZ_COLLIDE;
    }
    idx = q - C;
    return FZ_PASS1;
}

constexpr int WARPS_PER_ITEM = THREADS / 32;

// Whether pass-1 item j at position q of the sequence has a collision of its
// neighbourhood (the largest slot `far` of its table row) placed after it.
__device__ __forceinline__ bool fz_far(int far, int q, int L)
{
    return fz_pos_collide(PARTS * far + PARTS - 1, L) > q;
}

template <bool TAU1>
__global__ void __launch_bounds__(THREADS, 2) k_fused2(KParams kp)
{
    Ctrl *ctrl = kp.ctrl;
    const int tid = threadIdx.x, lane = tid & 31;
    const int step = *(volatile const int *)&ctrl->step;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    const bool run = *(volatile int *)&ctrl->status == 0 && in_range(kp, n, (long long)kp.capacity + 1, 7);
    const int C = run ? n * PARTS : 0;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;  // read by the collision
    float *wr = kp.f + (size_t)(par ^ 1) * kp.buf_stride;   // its output, read by pass 1
    // arrival counters of this launch, and the other parity's (cleared for
    // the next launch)
    int *cnt = kp.cflag + (size_t)par * kp.capacity * PARTS;
    int *cnt_next = kp.cflag + (size_t)(par ^ 1) * kp.capacity * PARTS;
    const int G = gridDim.x;
    int L = PARTS * (*(volatile int *)&ctrl->fz_dist + 1) + G;
    L = min(L, kp.fz_max_lag > 0 ? kp.fz_max_lag : FZ_MAX_LAG);
    L = max(0, min(L, C));
    if (run && blockIdx.x == 0 && tid == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    unsigned long long waited = 0, deferred = 0;  // lane 0 of warp 0: statistics
    // This warp's part of the last collision item, not yet counted: it is
    // counted once the next item's loads are consumed, when its stores have
    // long reached L2 and the fence before the count costs little.
    int pending = -1;
    auto publish = [&]() {
        if (pending >= 0) {
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicAdd(cnt + pending, 1);
            }
            pending = -1;
        }
    };

    // Pass 1 of item idx after its neighbourhood's collisions (all lanes of
    // the warp call).  `ready`: the counters were already seen complete.
    auto pass1 = [&](int idx, int row, uint32_t bits, bool ready, auto &&hook) {
        publish();  // never wait while holding an uncounted collision part
        bool ok = true, w = false;
        if (!__all_sync(FULL, ready) && row >= 0) {
#pragma unroll
            for (int p = 0; p < PARTS; ++p) {
                const int *fl = cnt + PARTS * row + p;
                for (long long it = 0; ld_relaxed(fl) < WARPS_PER_ITEM; ++it) {
                    w = true;
                    // give up after the poll limit, or once the launch has
                    if (it > kp.barrier_spins ||
                        ((it & 255) == 255 && *(volatile int *)&ctrl->status != 0)) {
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
                if (!ok) break;
            }
        }
        __syncwarp();  // the lanes' observations order every lane's loads below
        ok = __all_sync(FULL, ok);
        if (__any_sync(FULL, w) && tid == 0) ++waited;
        if (!ok) {
            if (lane == 0) atomicCAS(&ctrl->status, 0, LBM_ETIMEOUT);
            return;
        }
        macro2_item<true>(kp, ctrl, wr, par ^ 1, n, idx / PARTS, (idx % PARTS) * THREADS + tid, row, bits,
                          kp.progressive, false, float2{}, hook);
    };

    const int total = 2 * C;
    int q = blockIdx.x;
    int idx0;
    int next_row = SOLIDBLK;
    uint32_t next_bits = 1u;
    if (q < total) {
        fz_item(q, C, L, idx0);
        next_row = nbr_row_lane(kp, idx0 / PARTS);
        next_bits = kp.nbits[(size_t)(idx0 / PARTS) * CELLS + (idx0 % PARTS) * THREADS + tid];
    }
    // counters of the next pass-1 item's neighbourhood, read half an item
    // ahead (once its table row is in): complete counters stay complete
    bool next_ready = false;
    for (; q < total; q += G) {
        int idx;
        const int kind = fz_item(q, C, L, idx);
        const int row = next_row;
        const uint32_t bits = next_bits;
        const bool ready = next_ready;
        next_ready = false;
        int i2 = 0, kind2 = -1;
        if (q + G < total) {
            kind2 = fz_item(q + G, C, L, i2);
            next_row = nbr_row_lane(kp, i2 / PARTS);
            next_bits = kp.nbits[(size_t)(i2 / PARTS) * CELLS + (i2 % PARTS) * THREADS + tid];
        }
        // after the current item's loads: count the last collision part,
        // look at the next pass-1 item's counters
        auto hook = [&]() {
            publish();
            if (kind2 == FZ_PASS1) {
                bool r = true;
                if (next_row >= 0) {
#pragma unroll
                    for (int p = 0; p < PARTS; ++p) r = r && ld_relaxed(cnt + PARTS * next_row + p) >= WARPS_PER_ITEM;
                }
                next_ready = r;
            }
        };
        // (warp-uniform: lane 0's reading) the launch gave up
        if (__shfl_sync(FULL, *(volatile int *)&ctrl->status, 0) != 0) continue;
        if (kind == FZ_COLLIDE) {
            if (tid == 0) cnt_next[idx] = 0;
            collide2_item<TAU1>(kp, rd, wr, idx / PARTS, (idx % PARTS) * THREADS + tid, row, bits, nullptr,
                                hook);
            pending = idx;
        } else if (fz_far(__reduce_max_sync(FULL, row), q, L)) {
            if (tid == 0) ++deferred;  // redone below (lane 13 of row holds the slot itself)
        } else {
            pass1(idx, row, bits, ready, hook);
        }
    }
    publish();
    // the skipped pass-1 items of this CTA, every collision now placed before them
    for (q = blockIdx.x; q < total; q += G) {
        int idx;
        if (fz_item(q, C, L, idx) != FZ_PASS1) continue;
        const int row = nbr_row_lane(kp, idx / PARTS);
        if (!fz_far(__reduce_max_sync(FULL, row), q, L)) continue;
        if (__shfl_sync(FULL, *(volatile int *)&ctrl->status, 0) != 0) break;
        pass1(idx, row, kp.nbits[(size_t)(idx / PARTS) * CELLS + (idx % PARTS) * THREADS + tid], false,
              NoHook{});
    }
    if (tid == 0) {
        if (waited) atomicAdd(&ctrl->fz_waited, waited);
        if (deferred) atomicAdd(&ctrl->fz_deferred, deferred);
    }
    // the last CTA renumbers the next step's candidates and advances the step
    __shared__ int last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(&ctrl->collide_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (kp.progressive) order_candidates(kp, step + 1);
    __syncthreads();
    if (tid == 0) {
        ctrl->collide_done = 0u;
        if (__ldcg(&ctrl->status) == 0) ctrl->step = step + 1;
        __threadfence();
    }
}

// ---- A-A streaming: the two passes (FP32, two components) -------------------
// As k_macro2 / k_collide2 with the A-A addressing above; the kind of step
// (neighbour or local) follows the step count on the device, so captured
// launches replay correctly.

template <bool LOCAL>
__device__ __forceinline__ void macro_aa_body(const KParams &kp, int step, int criterion)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const int total = n * PARTS;
    const int ns = ctrl->n_sorted;  // work items below ns * PARTS visit kp.order
    auto slot_of_item = [&](int i) { return i / PARTS < ns ? kp.order[i / PARTS] : i / PARTS; };
    int it = blockIdx.x;
    int next_slot = it < total ? slot_of_item(it) : 0;
    int next_row = it < total ? nbr_row_lane(kp, next_slot) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)next_slot * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = next_slot;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, next_row);
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_slot = slot_of_item(it2);
            next_row = nbr_row_lane(kp, next_slot);
            next_bits = kp.nbits[(size_t)next_slot * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        const bool live = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 2))) continue;
        if (!criterion || wn.amb == 0u) {
            // warp-uniform: nothing for the criterion to test, only the
            // densities are needed (summed in the order of Moments2)
            float2 rho = make_float2(0.f, 0.f);
            pull2_aa<LOCAL>(kp, wn, slot, c, lx, ly, lz, bits, live, 0u,
                            [&]<int I>(float2 v) { rho = add2(rho, v); });
            kp.mac[(size_t)slot * CELLS + c] =
                live ? mac_pack(rho.x, psi_of(kp, rho.x), rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        Moments2 m;
        pull2_aa<LOCAL>(kp, wn, slot, c, lx, ly, lz, bits, live, 0u,
                        [&]<int I>(float2 v) { m.template add<I>(v); });
        const float2 inv = make_float2(1.f / m.rho.x, 1.f / m.rho.y);
        float u[2][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float2 ud = mul2(m.j[d], inv);
            u[0][d] = ud.x;
            u[1][d] = ud.y;
        }
        kp.mac[(size_t)slot * CELLS + c] =
            live ? mac_pack(m.rho.x, psi_of(kp, m.rho.x), m.rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (criterion) criterion_mark<2>(kp, ctrl, par, n, slot, c, wn, live && !held, u);
    }
}

__global__ void __launch_bounds__(THREADS, 4) k_macro_aa(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    if (step & 1)
        macro_aa_body<true>(kp, step, criterion);
    else
        macro_aa_body<false>(kp, step, criterion);
    if (criterion) order_tail(kp, step);
}

// The collision writes every non-solid cell: fluid cells their new
// populations, held cells their constants (the locations change from step
// to step); in local steps solid cells also complete sectors, as in
// k_collide2.  No lane leaves early: the write addresses of neighbour steps
// come from shuffles.
template <bool LOCAL, bool TAU1>
__device__ __forceinline__ void collide_aa_body(const KParams &kp, int step)
{
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n_old = ctrl->n_active[par];
    const int n = ctrl->n_active[par ^ 1];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 7)) return;
    float *A = kp.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    const int total = n * PARTS;
    const int ns = ctrl->n_sorted;  // work items below ns * PARTS visit kp.order
    auto slot_of_item = [&](int i) { return i / PARTS < ns ? kp.order[i / PARTS] : i / PARTS; };
    int it = blockIdx.x;
    int next_slot = it < total ? slot_of_item(it) : 0;
    int next_row = it < total ? nbr_row_lane(kp, next_slot) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)next_slot * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = next_slot;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, next_row);
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_slot = slot_of_item(it2);
            next_row = nbr_row_lane(kp, next_slot);
            next_bits = kp.nbits[(size_t)next_slot * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        const bool nonsolid = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        const bool live = nonsolid && !held;
        // blocks created in this step: ambient sources of a local step
        const unsigned fresh = LOCAL ? __ballot_sync(FULL, wn.slot >= n_old) : 0u;
        const bool row_live = row_has(nonsolid);  // every lane takes part
        const bool fill = LOCAL && (bits & 1u) && row_live;
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 8))) continue;
        Moments2 m;
        float2 fin[TAU1 ? 1 : Q];
        pull2_aa<LOCAL>(kp, wn, slot, c, lx, ly, lz, bits, nonsolid, fresh, [&]<int I>(float2 v) {
            m.template add<I>(v);
            if constexpr (!TAU1) fin[I] = v;
        });
        const float2 rho = m.rho;
        const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
        float2 u[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = mul2(m.j[d], inv);
        float2 F[3];
        forces2<2>(kp, wn, 0u, slot, c, lx, ly, lz, bits, live, rho, F);
        float2 v[3], nv[3], nu[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = fma2(F[d], inv, u[d]);
            nv[d] = sub2(make_float2(0.f, 0.f), v[d]);
            nu[d] = sub2(make_float2(0.f, 0.f), u[d]);
        }
        const float2 one = splat(1.f);
        const float2 cv = fma2(splat(-1.5f), fma2(v[0], v[0], fma2(v[1], v[1], mul2(v[2], v[2]))), one);
        const float2 cu = fma2(splat(-1.5f), fma2(u[0], u[0], fma2(u[1], u[1], mul2(u[2], u[2]))), one);
        float2 wrho[3];
        Unroll<0, 3>::run([&]<int K>() {
            constexpr int I = K == 0 ? 0 : (K == 1 ? 1 : 5);
            wrho[K] = mul2(splat(wgt(I)), rho);
        });
        const float2 relax = splat(1.f - kp.omega);
        float2 moving = make_float2(0.f, 0.f);
        const uint32_t own = (uint32_t)slot * (uint32_t)kp.slot_floats + (uint32_t)c;
        const bool store = nonsolid || fill;
        const float *hc = kp.held_f;
        if (held) hc += (size_t)kp.held_rank[kp.block_of[slot]] * kp.slot_floats + c;
        // the 18 moving populations (Eqs. 10-12); the rest population from
        // the mass balance sum_i f_i = rho (see k_collide)
        Unroll<1, Q>::run([&]<int I>() {
            const float2 ev = edot<I>(v, nv);
            float2 f = mul2(wrho[wclass(I)], fma2(ev, fma2(ev, splat(4.5f), splat(3.f)), cv));
            if constexpr (!TAU1) {
                const float2 eu = edot<I>(u, nu);
                const float2 e0 = mul2(wrho[wclass(I)], fma2(eu, fma2(eu, splat(4.5f), splat(3.f)), cu));
                f = fma2(relax, sub2(fin[I], e0), f);
            }
            moving = add2(moving, f);
            const uint32_t d = aa_dst<LOCAL, I>(wn, own, lx, ly, lz, bits);
            if (store) {
                A[d] = live ? f.x : (held ? __ldg(hc + I * CELLS) : 0.f);
                A[d + Q * CELLS] = live ? f.y : (held ? __ldg(hc + (Q + I) * CELLS) : 0.f);
            }
        });
        const float2 rest = sub2(rho, moving);
        if (store) {
            A[own] = live ? rest.x : (held ? __ldg(hc) : 0.f);
            A[own + Q * CELLS] = live ? rest.y : (held ? __ldg(hc + Q * CELLS) : 0.f);
        }
        (void)cu;
        if (live && kp.progressive && (reach_bits(lx, ly, lz) & wn.amb)) {
            float *up = kp.uprev + (size_t)slot * 2 * 3 * CELLS + c;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                up[d * CELLS] = u[d].x;
                up[(3 + d) * CELLS] = u[d].y;
            }
        }
    }
}

template <bool TAU1>
__global__ void __launch_bounds__(THREADS, 3) k_collide_aa(KParams kp)
{
    const int step = *(volatile const int *)&kp.ctrl->step;
    if (step & 1)
        collide_aa_body<true, TAU1>(kp, step);
    else
        collide_aa_body<false, TAU1>(kp, step);
    step_done(kp.ctrl, step);
}

// ---- TMA-staged step kernels (FP32, two components) -------------------------
// One CTA of 512 threads per SM works on one block at a time: the block's
// populations (both components, 77.8 KB, contiguous in the read buffer)
// arrive in shared memory with one bulk copy (cp.async.bulk), double
// buffered, so that the next block's copy is in flight while the current
// one is processed.  Pulls from inside the block read shared memory; only
// cells pulling across a face read the neighbour block in global memory.
// Same arithmetic in the same order as k_macro2 / k_collide2.
constexpr int TMA_THREADS = CELLS;
constexpr uint32_t SLOT2_BYTES = 2u * Q * CELLS * 4u;
constexpr size_t TMA_SMEM = 2 * (size_t)SLOT2_BYTES + 64;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for a phase of an mbarrier
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long spins)
{
    for (long long i = 0; i < spins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The block loop: cell(slot, c, stage) for every meshed slot, c the thread's
// cell, stage its block's populations ([comp][dir][cell] floats).  Only
// thread 0 issues copies and waits (a bounded wait: on time-out the status
// becomes LBM_ETIMEOUT, thread 0 waits again for its copies in flight, and
// the whole CTA returns together).
template <class Cell>
__device__ __forceinline__ void staged_blocks(const KParams &kp, const float *rd, int n, Cell &&cell)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int arrived;
    float *stage0 = reinterpret_cast<float *>(smem_raw);
    float *stage1 = reinterpret_cast<float *>(smem_raw + SLOT2_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + 2 * (size_t)SLOT2_BYTES);
    const int G = gridDim.x;
    int b = blockIdx.x;
    if (b >= n) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) bulk_load(stage0, rd + (size_t)b * kp.slot_floats, SLOT2_BYTES, &bar[0]);
    for (int k = 0; b < n; ++k, b += G) {
        const int s = k & 1;
        const int bn = b + G;
        if (threadIdx.x == 0) {
            if (bn < n) {
                fence_proxy_async();
                bulk_load(s ? stage0 : stage1, rd + (size_t)bn * kp.slot_floats, SLOT2_BYTES, &bar[s ^ 1]);
            }
            arrived = mbar_wait(&bar[s], (unsigned)(k >> 1) & 1u, kp.barrier_spins) ? 1 : 0;
            if (!arrived) {
                atomicCAS(&kp.ctrl->status, 0, LBM_ETIMEOUT);
                mbar_wait(&bar[s], (unsigned)(k >> 1) & 1u, kp.barrier_spins);
                if (bn < n) mbar_wait(&bar[s ^ 1], (unsigned)((k + 1) >> 1) & 1u, kp.barrier_spins);
            }
        }
        __syncthreads();
        if (!arrived) return;
        cell(b, (int)threadIdx.x, s ? stage1 : stage0);
        __syncthreads();  // the stage is free for the copy issued next iteration
    }
}

// pull2_f32 with the block's own populations in shared memory (st).
template <class Sink>
__device__ __forceinline__ void pull2_staged(const WarpNbr &wn, const float *rd, const float *st, int c,
                                             uint32_t bits, bool live, Sink &&sink)
{
    const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
    const bool held = (bits >> HELD_BIT) & 1u;
    uint32_t off[Q];
    uint32_t inside = 0;  // bit I: population I comes from the stage
    Unroll<0, Q>::run([&]<int I>() {
        const int sx = lx - cx(I), sy = ly - cy(I), sz = lz - cz(I);
        const int k = nbk(sx, sy, sz), lc = lcell(sx, sy, sz);
        const uint32_t base = __shfl_sync(FULL, wn.fbase, k);
        const bool bounce = (bits >> I) & 1u;
        const bool in = held || bounce || k == 13;
        off[I] = held ? (uint32_t)(I * CELLS + c)
                      : (bounce ? (uint32_t)(opp(I) * CELLS + c)
                                : (k == 13 ? (uint32_t)(I * CELLS + lc) : base + (uint32_t)(I * CELLS + lc)));
        inside |= (uint32_t)in << I;
    });
    float2 v[Q];
    Unroll<0, Q>::run([&]<int I>() {
        if (!live)
            v[I] = make_float2(0.f, 0.f);
        else if ((inside >> I) & 1u)
            v[I] = make_float2(st[off[I]], st[off[I] + Q * CELLS]);
        else
            v[I] = make_float2(__ldg(rd + off[I]), __ldg(rd + off[I] + Q * CELLS));
    });
    sink.template operator()<0>(v[0]);
    Unroll<0, NPAIR>::run([&]<int P>() {
        sink.template operator()<pair_rep(P)>(v[pair_rep(P)]);
        sink.template operator()<opp(pair_rep(P))>(v[opp(pair_rep(P))]);
    });
}

__device__ __forceinline__ void macro2_staged_body(const KParams &kp, int step, int criterion)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    staged_blocks(kp, rd, n, [&](int slot, int c, const float *st) {
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
        const bool live = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 2))) return;
        Moments2 m;
        pull2_staged(wn, rd, st, c, bits, live, [&]<int I>(float2 v) { m.template add<I>(v); });
        const float2 inv = make_float2(1.f / m.rho.x, 1.f / m.rho.y);
        float u[2][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float2 ud = mul2(m.j[d], inv);
            u[0][d] = ud.x;
            u[1][d] = ud.y;
        }
        kp.mac[(size_t)slot * CELLS + c] =
            live ? mac_pack(m.rho.x, psi_of(kp, m.rho.x), m.rho.y) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (criterion) criterion_mark<2>(kp, ctrl, par, n, slot, c, wn, live && !held, u);
    });
}

__global__ void __launch_bounds__(TMA_THREADS, 1) k_macro2_staged(KParams kp, int criterion)
{
    const int step = kp.ctrl->step;
    macro2_staged_body(kp, step, criterion);
    if (criterion) order_tail(kp, step);
}

template <bool TAU1>
__device__ __forceinline__ void collide2_staged_body(const KParams &kp, int step)
{
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 7)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    float *wr = kp.f + (size_t)(par ^ 1) * kp.buf_stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    staged_blocks(kp, rd, n, [&](int slot, int c, const float *st) {
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
        const bool live = !(bits & 1u) && !((bits >> HELD_BIT) & 1u);
        // every lane takes part in the ballot (it must not sit behind &&)
        const bool row_live = row_has(live);
        const bool fill = (bits & 1u) && row_live;  // solid cell completing a sector
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 8))) return;
        Moments2 m;
        float2 fin[TAU1 ? 1 : Q];
        pull2_staged(wn, rd, st, c, bits, live, [&]<int I>(float2 v) {
            m.template add<I>(v);
            if constexpr (!TAU1) fin[I] = v;
        });
        const float2 rho = m.rho;
        const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
        float2 u[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) u[d] = mul2(m.j[d], inv);
        float2 F[3];
        forces2<2>(kp, wn, 0u, slot, c, lx, ly, lz, bits, live, rho, F);
        if (!live && !fill) return;
        float2 v[3], nv[3], nu[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            v[d] = fma2(F[d], inv, u[d]);
            nv[d] = sub2(make_float2(0.f, 0.f), v[d]);
            nu[d] = sub2(make_float2(0.f, 0.f), u[d]);
        }
        const float2 one = splat(1.f);
        const float2 cv = fma2(splat(-1.5f), fma2(v[0], v[0], fma2(v[1], v[1], mul2(v[2], v[2]))), one);
        const float2 cu = fma2(splat(-1.5f), fma2(u[0], u[0], fma2(u[1], u[1], mul2(u[2], u[2]))), one);
        float2 wrho[3];
        Unroll<0, 3>::run([&]<int K>() {
            constexpr int I = K == 0 ? 0 : (K == 1 ? 1 : 5);
            wrho[K] = mul2(splat(wgt(I)), rho);
        });
        const float2 relax = splat(1.f - kp.omega);
        float2 moving = make_float2(0.f, 0.f);
        float *d0 = wr + (size_t)slot * kp.slot_floats + c;
        float *d1 = d0 + Q * CELLS;
        Unroll<1, Q>::run([&]<int I>() {
            const float2 ev = edot<I>(v, nv);
            float2 f = mul2(wrho[wclass(I)], fma2(ev, fma2(ev, splat(4.5f), splat(3.f)), cv));
            if constexpr (!TAU1) {
                const float2 eu = edot<I>(u, nu);
                const float2 e0 = mul2(wrho[wclass(I)], fma2(eu, fma2(eu, splat(4.5f), splat(3.f)), cu));
                f = fma2(relax, sub2(fin[I], e0), f);
            }
            moving = add2(moving, f);
            d0[I * CELLS] = live ? f.x : 0.f;
            d1[I * CELLS] = live ? f.y : 0.f;
        });
        const float2 rest = sub2(rho, moving);
        d0[0] = live ? rest.x : 0.f;
        d1[0] = live ? rest.y : 0.f;
        (void)cu;
        if (live && kp.progressive && (reach_bits(lx, ly, lz) & wn.amb)) {
            float *up = kp.uprev + (size_t)slot * 2 * 3 * CELLS + c;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                up[d * CELLS] = u[d].x;
                up[(3 + d) * CELLS] = u[d].y;
            }
        }
    });
}

template <bool TAU1>
__global__ void __launch_bounds__(TMA_THREADS, 1) k_collide2_staged(KParams kp)
{
    const int step = *(volatile const int *)&kp.ctrl->step;
    collide2_staged_body<TAU1>(kp, step);
    step_done(kp.ctrl, step);
}

// Pass 2 of a step in the deviation forms (as k_collide, paired arithmetic
// for the two components).  Every value
// is stored against the density its reader has now: the neighbour's mac of
// this step, the cell's own behind a solid cell and for the rest
// population.  Held cells write their constant equilibrium (density from
// mac, velocity from uprev).  With one component the second half of each
// word carries a dummy unit-density state.
template <int NC, bool TAU1, int ST>
__device__ __forceinline__ void collide_dev_body(const KParams &kp, int step)
{
    using S = Store<ST>;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 7)) return;
    const uint32_t *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
    uint32_t *wr = pops<ST>(kp) + (size_t)(par ^ 1) * kp.buf_stride;
    const uint32_t moff = (uint32_t)(par * kp.mac_stride);
    const float4 *mac_prev = kp.mac + (size_t)(par ^ 1) * kp.mac_stride;
    // the readers' density pairs of this thread's cell, kept by the force
    // gather (each thread reads back only its own column: no barrier)
    __shared__ float2 rn_s[Q][THREADS];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->cell_updates += (unsigned long long)n * CELLS;
        ctrl->fluid_updates += ctrl->fluid_active;
    }
    const int total = n * PARTS;
    int it = blockIdx.x;
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        DevItem cur;
        dev_item<ST>(kp, rd, mac_prev, it, next_row, next_bits, moff, cur);
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        // (every lane votes: the collective must not sit behind &&)
        const bool any_cell = __any_sync(FULL, !(cur.bits & 1u));
        if (cur.ok && any_cell) {  // skip warps of solid cells only
            const int slot = cur.slot, c = cur.c;
            const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
            const uint32_t bits = cur.bits;
            const bool nonsolid = !(bits & 1u);
            const bool held = (bits >> HELD_BIT) & 1u;
            const bool live = nonsolid && !held;
            float2 wref[3], famb[3];
            amb_and_refs(kp, cur.ref, wref, famb);
            Moments2 m;
            float2 fin[TAU1 ? 1 : Q];
            dev_consume2<ST>(cur.L, wref, famb, [&]<int I>(float2 v) {
                m.template add<I>(v);
                if constexpr (!TAU1) fin[I] = v;
            });
            float2 rho = m.rho;
            if (NC == 1) rho.y = 1.f;
            float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
            float2 u[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) u[d] = mul2(m.j[d], inv);
            if (held) {
                rho = cur.ref;
                if (NC == 1) rho.y = 1.f;
                const float *up = kp.uprev + (size_t)slot * NC * 3 * CELLS + c;
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    u[d] = make_float2(up[d * CELLS], NC == 2 ? up[(3 + d) * CELLS] : 0.f);
                inv = make_float2(0.f, 0.f);  // no force term
            }
            if (NC == 1)
#pragma unroll
                for (int d = 0; d < 3; ++d) u[d].y = 0.f;
            float2 F[3];
            forces2<NC>(kp, cur.wn, moff, slot, c, lx, ly, lz, bits, nonsolid, rho, F, &rn_s[0][threadIdx.x]);
            // Eqs. 10-12 with tau = 1 (f* = f_eq(rho, u + F / rho)), else
            // f* = f_eq(rho, u + F / rho) + (1 - 1/tau) (f - f_eq(rho, u));
            // every lane runs it (its shuffles need the whole warp), solid
            // cells store nothing
            float2 v[3], nv[3], nu[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = fma2(F[d], inv, u[d]);
                nv[d] = sub2(make_float2(0.f, 0.f), v[d]);
                nu[d] = sub2(make_float2(0.f, 0.f), u[d]);
            }
            const float2 one = splat(1.f);
            const float2 cv = fma2(splat(-1.5f), fma2(v[0], v[0], fma2(v[1], v[1], mul2(v[2], v[2]))), one);
            const float2 cu = fma2(splat(-1.5f), fma2(u[0], u[0], fma2(u[1], u[1], mul2(u[2], u[2]))), one);
            float2 wrho[3];
            Unroll<0, 3>::run([&]<int K>() {
                constexpr int I = K == 0 ? 0 : (K == 1 ? 1 : 5);
                wrho[K] = mul2(splat(wgt(I)), rho);
            });
            const float2 relax = splat(held ? 0.f : 1.f - kp.omega);
            float2 moving = make_float2(0.f, 0.f);
            uint32_t *dst = wr + (size_t)slot * kp.slot_floats + c;
            Unroll<1, Q>::run([&]<int I>() {
                const float2 ev = edot<I>(v, nv);
                float2 f = mul2(wrho[wclass(I)], fma2(ev, fma2(ev, splat(4.5f), splat(3.f)), cv));
                if constexpr (!TAU1) {
                    const float2 eu = edot<I>(u, nu);
                    const float2 e0 = mul2(wrho[wclass(I)], fma2(eu, fma2(eu, splat(4.5f), splat(3.f)), cu));
                    f = fma2(relax, sub2(fin[I], e0), f);
                }
                // the reader's density: the neighbour's (kept by the force
                // gather), or the cell's own
                const float2 rr = nonsolid ? rn_s[I][threadIdx.x] : rho;
                const float2 d = fma2(splat(-wgt(I)), rr, f);
                const uint32_t h = S::enc2(d.x, d.y);
                if (nonsolid) dst[I * CELLS] = h;
                // the value its reader will decode, rounding included
                moving = add2(moving, add2(S::dec2(h), mul2(splat(wgt(I)), rr)));
            });
            // rest population from the mass balance sum_i f_i = rho over the
            // stored values: the cell's 16-bit rounding leaves its mass unchanged
            const float2 d0 = fma2(splat(-wgt(0)), rho, sub2(rho, moving));
            if (nonsolid) dst[0] = S::enc2(d0.x, d0.y);
            (void)cu;
            if (live && kp.progressive && (reach_bits(lx, ly, lz) & cur.wn.amb)) {
                float *up = kp.uprev + (size_t)slot * NC * 3 * CELLS + c;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    up[d * CELLS] = u[d].x;
                    if (NC == 2) up[(3 + d) * CELLS] = u[d].y;
                }
            }
        }
    }
}

template <int NC, bool TAU1, int ST>
__global__ void __launch_bounds__(THREADS, DEV_COLLIDE_MIN_CTAS) k_collide_dev(KParams kp)
{
    const int step = *(volatile const int *)&kp.ctrl->step;
    collide_dev_body<NC, TAU1, ST>(kp, step);
    step_done(kp.ctrl, step);
}

// Macroscopic output of one component for slots [slot0, slot0 + nslots):
// out[slot - slot0][4][CELLS] = rho, ux, uy, uz, velocity u + F / (2 rho)
// at fluid cells (the exact-difference forcing's physical velocity), own
// moments at held cells, zeros at solid cells.
// Expects mac of this step (k_macro without the criterion).
template <int NC, int ST>
__global__ void __launch_bounds__(THREADS) k_output(KParams kp, int rdbuf, int comp, int slot0,
                                                    int nslots, float *out)
{
    using S = Store<ST>;
    const typename S::T *rd = pops<ST>(kp) + (size_t)rdbuf * kp.buf_stride;
    const uint32_t moff = S::DEV ? (uint32_t)(rdbuf * kp.mac_stride) : 0u;
    const float4 *mac_prev = kp.mac + (size_t)(rdbuf ^ 1) * kp.mac_stride;
    for (int it = blockIdx.x; it < nslots * PARTS; it += gridDim.x) {
        const int r = it / PARTS;
        const int slot = slot0 + r;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot), moff);
        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
        const bool live = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        float ref[2] = {0.f, 0.f};
        if constexpr (S::DEV) {
            if (live) {
                const float4 p = __ldg(mac_prev + (size_t)slot * CELLS + c);
                ref[0] = p.x;
                ref[1] = p.y;
            }
        }
        Moments m;
        pull_state<NC, ST>(kp, wn, rd, rdbuf, slot, c, lx, ly, lz, bits, live, ref,
                           [&]<int I>(int a, float v) { m.template add<I>(a, v); });
        float rho[2] = {m.rho[0], m.rho[1]};
        float F[2][3];
        forces<NC>(kp, wn, moff, slot, c, lx, ly, lz, bits, live && !held, rho, F);
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
            const int a = comp;
            const float inv = 1.f / rho[a];
            o[0] = rho[a];
            o[1] = m.j[a][0] * inv;
            o[2] = m.j[a][1] * inv;
            o[3] = m.j[a][2] * inv;
            if (!held) {
                const float h = 0.5f * inv;
                o[1] += F[a][0] * h;
                o[2] += F[a][1] * h;
                o[3] += F[a][2] * h;
            } else if (S::DEV) {
                const float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                o[0] = ref[a];
                o[1] = up[0];
                o[2] = up[CELLS];
                o[3] = up[2 * CELLS];
            }
        }
        float *dst = out + (size_t)r * 4 * CELLS + c;
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q * CELLS] = o[q];
    }
}

// The stored populations of one cell of buffer rdbuf as FP32 values (the
// deviation forms add their readers' references back, from the mac of the
// step that wrote them); zeros at solid cells.  All lanes of the warp call.
template <int ST>
__device__ __forceinline__ void stored_cell(const KParams &kp, int rdbuf, int slot, int c,
                                            float out[2][Q])
{
    using S = Store<ST>;
    const typename S::T *src = pops<ST>(kp) + (size_t)rdbuf * kp.buf_stride +
                               (size_t)slot * kp.slot_floats + c;
    const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
    const bool live = !(bits & 1u);
    float rdst[2][Q];
    if constexpr (S::DEV) {
        const float4 *mref = kp.mac + (size_t)(rdbuf ^ 1) * kp.mac_stride;
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
        const float4 m = live ? __ldg(mref + (size_t)slot * CELLS + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float own[2] = {m.x, m.y};
        reader_refs<2>(wn, mref, lx_of(c), ly_of(c), lz_of(c), bits, live, own, rdst);
    }
    if constexpr (S::DEV) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float2 x = S::dec2(__ldg(src + i * CELLS));
            out[0][i] = live ? __fmaf_rn(wgt(i), rdst[0][i], x.x) : 0.f;
            out[1][i] = live ? __fmaf_rn(wgt(i), rdst[1][i], x.y) : 0.f;
        }
    } else if (kp.aa) {
        // A-A: where the last step left each outgoing value (rdbuf is the
        // parity of the next step; the initial state is laid out as after a
        // local step)
        const uint32_t own = (uint32_t)slot * (uint32_t)kp.slot_floats + (uint32_t)c;
        const int lx = lx_of(c), ly = ly_of(c), lz = lz_of(c);
        if (rdbuf == 0) {
            Unroll<0, Q>::run([&]<int I>() {
                const uint32_t d = aa_dst<true, I>(WarpNbr{}, own, lx, ly, lz, bits);
                out[0][I] = live ? __ldg(kp.f + d) : 0.f;
                out[1][I] = live ? __ldg(kp.f + d + Q * CELLS) : 0.f;
            });
        } else {
            const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
            Unroll<0, Q>::run([&]<int I>() {
                const uint32_t d = aa_dst<false, I>(wn, own, lx, ly, lz, bits);
                out[0][I] = live ? __ldg(kp.f + d) : 0.f;
                out[1][I] = live ? __ldg(kp.f + d + Q * CELLS) : 0.f;
            });
        }
    } else {
        for (int a = 0; a < kp.ncomp; ++a)
#pragma unroll
            for (int i = 0; i < Q; ++i) out[a][i] = __ldg(src + (a * Q + i) * CELLS);
    }
}

// FP64 mass: per-slot partial sums over non-solid cells, then one CTA adds
// the partials in a fixed order.
template <int ST>
__global__ void __launch_bounds__(CELLS) k_mass_partial(KParams kp, int rdbuf, int n,
                                                        double *partial)
{
    __shared__ double red[CELLS / 32][2];
    const int c = threadIdx.x;
    for (int slot = blockIdx.x; slot < n; slot += gridDim.x) {
        const bool solid = kp.nbits[(size_t)slot * CELLS + c] & 1u;
        float f[2][Q];
        stored_cell<ST>(kp, rdbuf, slot, c, f);
        double m[2] = {0.0, 0.0};
        for (int a = 0; a < kp.ncomp; ++a) {
            if (solid) continue;
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += (double)f[a][i];
            m[a] = acc;
        }
        for (int a = 0; a < 2; ++a)
            for (int o = 16; o > 0; o >>= 1) m[a] += __shfl_down_sync(FULL, m[a], o);
        if ((c & 31) == 0) {
            red[c >> 5][0] = m[0];
            red[c >> 5][1] = m[1];
        }
        __syncthreads();
        if (c < 2) {
            double t = 0.0;
            for (int w = 0; w < CELLS / 32; ++w) t += red[w][c];
            partial[(size_t)slot * 2 + c] = t;
        }
        __syncthreads();
    }
}

// The populations of one slot, decoded to FP32: out[ncomp][Q][CELLS].
template <int ST>
__global__ void __launch_bounds__(CELLS) k_block_pops(KParams kp, int rdbuf, int slot, float *out)
{
    const int c = threadIdx.x;
    float f[2][Q];
    stored_cell<ST>(kp, rdbuf, slot, c, f);
    for (int a = 0; a < kp.ncomp; ++a)
#pragma unroll
        for (int i = 0; i < Q; ++i) out[(a * Q + i) * CELLS + c] = f[a][i];
}

// Features of the listed frontier blocks (include/lbm.h, proposer): one CTA
// per block; warps 0-5 take the faces -x, +x, -y, +y, -z, +z and pull the 64
// cells of the meshed neighbour that touch the block (held and solid cells
// left out), warp 6 the neighbour flags.  par: the read buffer.  Only slots
// below *nsnap, a count of meshed blocks taken between two steps, are read:
// their table rows are complete, while a slot handed out later may not be
// yet (this kernel may run beside the step kernels).
template <int NC, int ST>
__global__ void __launch_bounds__(THREADS) k_features(KParams kp, int par, const int *nsnap,
                                                      const int *list, const int *count, float *feat)
{
    if constexpr (BX == 8 && BY == 8 && BZ == 8) {  // the features are defined on 8 x 8 faces
        using S = Store<ST>;
        __shared__ float acc[6][4];  // per face: sum rho0, sum rho1, cells, flux
        const typename S::T *rd = pops<ST>(kp) + (size_t)par * kp.buf_stride;
        const float4 *mac_prev = kp.mac + (size_t)(par ^ 1) * kp.mac_stride;
        const int n = *count;
        const int nmesh = *nsnap;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int b = blockIdx.x; b < n; b += gridDim.x) {
            const int gid = list[b];
            float *out = feat + (size_t)b * LBM_MLP_IN;
            if (warp < 6) {
                const int axis = warp >> 1, sgn = (warp & 1) ? 1 : -1;  // neighbour at gid + sgn e_axis
                const int k = 13 + sgn * (axis == 0 ? 1 : (axis == 1 ? 3 : 9));
                const int nid = neighbour_of(kp, gid, k);
                const int slot = nid >= 0 ? kp.slot_of[nid] : SOLIDBLK;
                float r0 = 0.f, r1 = 0.f, cnt = 0.f, flux = 0.f;
                if (slot >= 0 && slot < nmesh) {
                    const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
                    const int layer = sgn < 0 ? 7 : 0;  // the neighbour's cells touching the block
    #pragma unroll 1
                    for (int pass = 0; pass < 2; ++pass) {
                        const int idx = pass * 32 + lane, u = idx & 7, v = idx >> 3;
                        const int lx = axis == 0 ? layer : u, ly = axis == 1 ? layer : (axis == 0 ? u : v),
                                  lz = axis == 2 ? layer : v;
                        const int c = lx | (ly << 3) | (lz << 6);
                        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
                        const bool use = !(bits & 1u) && !((bits >> HELD_BIT) & 1u);
                        float ref[2] = {0.f, 0.f};
                        if (S::DEV && use) {
                            const float4 m = __ldg(mac_prev + (size_t)slot * CELLS + c);
                            ref[0] = m.x;
                            ref[1] = m.y;
                        }
                        Moments m;
                        pull_state<NC, ST>(kp, wn, rd, par, slot, c, lx, ly, lz, bits, use, ref,
                                           [&]<int I>(int a, float f) { m.template add<I>(a, f); });
                        if (use) {
                            r0 += m.rho[0];
                            r1 += NC == 2 ? m.rho[1] : 0.f;
                            cnt += 1.f;
                            // into the block: along -sgn e_axis
                            const float j = m.j[0][axis] + (NC == 2 ? m.j[1][axis] : 0.f);
                            flux -= (float)sgn * j;
                        }
                    }
                }
    #pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r0 += __shfl_xor_sync(FULL, r0, o);
                    r1 += __shfl_xor_sync(FULL, r1, o);
                    cnt += __shfl_xor_sync(FULL, cnt, o);
                    flux += __shfl_xor_sync(FULL, flux, o);
                }
                if (lane == 0) {
                    acc[warp][0] = r0;
                    acc[warp][1] = r1;
                    acc[warp][2] = cnt;
                    acc[warp][3] = flux;
                }
            } else if (warp == 6 && lane < 27 && lane != 13) {
                const int nid = neighbour_of(kp, gid, lane);
                // (a candidate of the next step, already marked, has a slot
                // at or beyond nmesh: not meshed yet)
                const int ns = nid >= 0 ? kp.slot_of[nid] : SOLIDBLK;
                out[8 + lane - (lane > 13 ? 1 : 0)] = (ns >= 0 && ns < nmesh) ? 1.f : 0.f;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                float r0 = 0.f, r1 = 0.f, cnt = 0.f;
                for (int f = 0; f < 6; ++f) {
                    r0 += acc[f][0];
                    r1 += acc[f][1];
                    cnt += acc[f][2];
                    out[2 + f] = acc[f][3];
                }
                out[0] = cnt > 0.f ? r0 / cnt : kp.rho_amb[0];
                out[1] = cnt > 0.f ? r1 / cnt : kp.rho_amb[1];
            }
            __syncthreads();
        }
    }
}

// ---- whole steps in one cooperative launch ----------------------------------

// Grid-wide barrier with a bounded wait: CTA leaders count in; the last one
// resets the count and advances the generation, the others poll it.  A
// wait that exceeds `spins` polls sets LBM_ETIMEOUT and gives up, so no
// launch can hang.  Returns false when the status is no longer 0.
__device__ __forceinline__ bool grid_sync(Ctrl *ctrl, unsigned expect, long long spins)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctrl->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&ctrl->bar_count, 1u) == expect - 1) {
            ctrl->bar_count = 0u;
            __threadfence();
            atomicAdd(&ctrl->bar_gen, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > spins) {
                    atomicCAS(&ctrl->status, 0, LBM_ETIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)&ctrl->status == 0;
}

// The phases of one storage form and component count.
template <int NC, bool TAU1, int ST>
struct Phases {
    static constexpr int MIN_CTAS = Store<ST>::DEV ? DEV_COLLIDE_MIN_CTAS : 2;
    __device__ __forceinline__ static void macro(const KParams &kp, int step, int crit, bool part_in)
    {
        if constexpr (Store<ST>::DEV)
            macro_dev_body<NC, ST>(kp, step, crit);
        else if constexpr (NC == 2)
            macro2_body(kp, step, crit, part_in);
        else
            macro_body<NC>(kp, step, crit);
    }
    __device__ __forceinline__ static void collide(const KParams &kp, int step)
    {
        if constexpr (Store<ST>::DEV) {
            collide_dev_body<NC, TAU1, ST>(kp, step);
        } else if constexpr (NC == 2) {
            if (kp.part_out)
                collide2_body<TAU1, true>(kp, step);
            else
                collide2_body<TAU1>(kp, step);
        } else {
            collide_body<NC, TAU1>(kp, step);
        }
    }
};

// nsteps steps: stream + moments (+ criterion), grid barrier, block
// creation, barrier, forces + collision, barrier; the same bodies as the
// per-phase launches, so the results are the same bit for bit.  The first
// pass 1 sums the density partials when kp.part_in says they are there,
// the others when the collisions write them (kp.part_out).
template <int NC, bool TAU1, int ST>
__global__ void __launch_bounds__(THREADS, (Phases<NC, TAU1, ST>::MIN_CTAS)) k_run(KParams kp, int nsteps,
                                                                              int progressive)
{
    using P = Phases<NC, TAU1, ST>;
    Ctrl *ctrl = kp.ctrl;
    int step = *(volatile int *)&ctrl->step;
    for (int k = 0; k < nsteps; ++k, ++step) {
        P::macro(kp, step, progressive, k == 0 ? kp.part_in != 0 : kp.part_out != 0);
        if (!grid_sync(ctrl, gridDim.x, kp.barrier_spins)) return;
        if (progressive) {
            if (blockIdx.x == 0) order_body(kp, step);
            if (!grid_sync(ctrl, gridDim.x, kp.barrier_spins)) return;
            activate_body<NC, ST>(kp, step);
            if (!grid_sync(ctrl, gridDim.x, kp.barrier_spins)) return;
        }
        P::collide(kp, step);
        if (!grid_sync(ctrl, gridDim.x, kp.barrier_spins)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->step = step + 1;
    }
}

// ---- launch wrappers of one storage form -------------------------------------

// Resident CTAs per SM of a kernel with SMEM bytes of dynamic shared
// memory (opted in above the default 48 KB), looked up once per process.
template <auto Kern, size_t SMEM = 0>
int occupancy()
{
    static int cached = 0;
    if (!cached) {
        if (SMEM > 48 * 1024) cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, Kern, THREADS, SMEM) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        cached = n > 0 ? n : 1;
    }
    return cached;
}

template <auto Kern, size_t SMEM = 0, class... A>
cudaError_t launch_persistent(int sms, cudaStream_t s, A... args)
{
    Kern<<<sms * occupancy<Kern, SMEM>(), THREADS, SMEM, s>>>(args...);
    return cudaGetLastError();
}

// Launch of the fused step: the resident CTAs less one when their number is
// even.  CTA g takes positions g, g + G, ... of a sequence that alternates
// collision and pass-1 items by position, so an odd G makes every CTA
// alternate too (an even G would give half the CTAs only collisions and the
// other half only pass-1 items, which then wait on them).
template <auto Kern, class... A>
cudaError_t launch_fused_grid(int sms, cudaStream_t s, A... args)
{
    int g = sms * occupancy<Kern>();
    if (g > 1 && (g & 1) == 0) g -= 1;
    Kern<<<g, THREADS, 0, s>>>(args...);
    return cudaGetLastError();
}

// Launch of a TMA-staged kernel: one CTA of TMA_THREADS per resident slot,
// TMA_SMEM bytes of dynamic shared memory (opted in once per kernel).
template <auto Kern, class... A>
cudaError_t launch_staged(int sms, cudaStream_t s, A... args)
{
    static int occ = 0;
    if (!occ) {
        cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, Kern, TMA_THREADS, TMA_SMEM) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        occ = n > 0 ? n : 1;
    }
    Kern<<<sms * occ, TMA_THREADS, TMA_SMEM, s>>>(args...);
    return cudaGetLastError();
}

template <int ST>
struct Launch {
    static cudaError_t init(const KParams &kp, const float *in_block, int slot0, int nslots, int grid,
                            cudaStream_t s)
    {
        if (nslots <= 0) return cudaSuccess;
        k_init<ST><<<grid, CELLS, 0, s>>>(kp, in_block, slot0, nslots);
        return cudaGetLastError();
    }
    static cudaError_t init_finish(const KParams &kp, int nslots, int sms, cudaStream_t s)
    {
        if constexpr (!Store<ST>::DEV) {
            return cudaSuccess;
        } else {
            if (nslots <= 0) return cudaSuccess;
            if (kp.ncomp == 2) return launch_persistent<k_init_dev<2, ST>>(sms, s, kp, nslots);
            return launch_persistent<k_init_dev<1, ST>>(sms, s, kp, nslots);
        }
    }
    static cudaError_t ambient_slot(const KParams &kp, cudaStream_t s)
    {
        k_ambient_slot<ST><<<1, CELLS, 0, s>>>(kp);
        return cudaGetLastError();
    }
    static cudaError_t macro(const KParams &kp, int step, int criterion, int sms, cudaStream_t s)
    {
        if constexpr (Store<ST>::DEV) {
            if (kp.ncomp == 2) return launch_persistent<k_macro_dev<2, ST>>(sms, s, kp, criterion);
            return launch_persistent<k_macro_dev<1, ST>>(sms, s, kp, criterion);
        } else {
            if (kp.aa) return launch_persistent<k_macro_aa>(sms, s, kp, criterion);
            if (kp.ncomp == 2 && kp.staged) return launch_staged<k_macro2_staged>(sms, s, kp, criterion);
            if (kp.ncomp == 2 && kp.part_in) {
                cudaError_t e = launch_persistent<k_macro2p>(sms, s, kp);
                if (e == cudaSuccess && kp.progressive) e = launch_persistent<k_macro2f>(sms, s, kp, criterion);
                return e;
            }
            if (kp.ncomp == 2) return launch_persistent<k_macro2>(sms, s, kp, criterion);
            return launch_persistent<k_macro<1>>(sms, s, kp, criterion);
        }
    }
    static cudaError_t activate(const KParams &kp, int step, int sms, cudaStream_t s)
    {
        // (the candidates were renumbered in block order by the pass-1 launch)
        if (kp.ncomp == 2)
            k_activate<2, ST><<<2 * sms, THREADS, 0, s>>>(kp);
        else
            k_activate<1, ST><<<2 * sms, THREADS, 0, s>>>(kp);
        return cudaGetLastError();
    }
    static cudaError_t collide(const KParams &kp, int step, int sms, cudaStream_t s)
    {
        const bool tau1 = kp.omega == 1.0f;
        if constexpr (Store<ST>::DEV) {
            if (kp.ncomp == 2) {
                if (tau1) return launch_persistent<k_collide_dev<2, true, ST>>(sms, s, kp);
                return launch_persistent<k_collide_dev<2, false, ST>>(sms, s, kp);
            }
            if (tau1) return launch_persistent<k_collide_dev<1, true, ST>>(sms, s, kp);
            return launch_persistent<k_collide_dev<1, false, ST>>(sms, s, kp);
        } else {
            if (kp.aa) {
                if (tau1) return launch_persistent<k_collide_aa<true>>(sms, s, kp);
                return launch_persistent<k_collide_aa<false>>(sms, s, kp);
            }
            if (kp.ncomp == 2 && kp.staged) {
                if (tau1) return launch_staged<k_collide2_staged<true>>(sms, s, kp);
                return launch_staged<k_collide2_staged<false>>(sms, s, kp);
            }
            if (kp.ncomp == 2 && kp.part_out) {
                if (tau1) return launch_persistent<k_collide2<true, true>, PART_SMEM>(sms, s, kp);
                return launch_persistent<k_collide2<false, true>, PART_SMEM>(sms, s, kp);
            }
            if (kp.ncomp == 2) {
                if (tau1) return launch_persistent<k_collide2<true, false>>(sms, s, kp);
                return launch_persistent<k_collide2<false, false>>(sms, s, kp);
            }
            if (tau1) return launch_persistent<k_collide<1, true>>(sms, s, kp);
            return launch_persistent<k_collide<1, false>>(sms, s, kp);
        }
    }
    static cudaError_t output(const KParams &kp, int rd, int comp, int slot0, int nslots, float *out,
                              int sms, cudaStream_t s)
    {
        if (nslots <= 0) return cudaSuccess;
        if (kp.ncomp == 2)
            return launch_persistent<k_output<2, ST>>(sms, s, kp, rd, comp, slot0, nslots, out);
        return launch_persistent<k_output<1, ST>>(sms, s, kp, rd, comp, slot0, nslots, out);
    }
    static cudaError_t mass_partial(const KParams &kp, int rd, int n, double *partial, int grid,
                                    cudaStream_t s)
    {
        if (n <= 0) return cudaSuccess;
        k_mass_partial<ST><<<grid, CELLS, 0, s>>>(kp, rd, n, partial);
        return cudaGetLastError();
    }
    static cudaError_t block_pops(const KParams &kp, int rd, int slot, float *out, cudaStream_t s)
    {
        k_block_pops<ST><<<1, CELLS, 0, s>>>(kp, rd, slot, out);
        return cudaGetLastError();
    }
    static cudaError_t features(const KParams &kp, int par, const int *nsnap, const int *list,
                                const int *count, float *feat, int sms, cudaStream_t s)
    {
        if (kp.ncomp == 2)
            k_features<2, ST><<<sms * 2, THREADS, 0, s>>>(kp, par, nsnap, list, count, feat);
        else
            k_features<1, ST><<<sms * 2, THREADS, 0, s>>>(kp, par, nsnap, list, count, feat);
        return cudaGetLastError();
    }
    template <int NC, bool TAU1>
    static cudaError_t run_on(const KParams &kp, int nsteps, int progressive, int sms, cudaStream_t s)
    {
        auto kern = k_run<NC, TAU1, ST>;
        // (the grid fits the residency with the partials' shared memory,
        // whether or not this launch writes them)
        constexpr size_t RUN_SMEM = !Store<ST>::DEV && NC == 2 ? PART_SMEM : 0;
        const int grid = sms * occupancy<k_run<NC, TAU1, ST>, RUN_SMEM>();
        KParams a = kp;
        void *args[] = {&a, &nsteps, &progressive};
        return cudaLaunchCooperativeKernel((const void *)kern, grid, THREADS, args, kp.part_out ? RUN_SMEM : 0,
                                           s);
    }
    static cudaError_t run(const KParams &kp, int nsteps, int progressive, int sms, cudaStream_t s)
    {
        if (nsteps <= 0) return cudaSuccess;
        const bool tau1 = kp.omega == 1.0f;
        if (kp.ncomp == 2)
            return tau1 ? run_on<2, true>(kp, nsteps, progressive, sms, s)
                        : run_on<2, false>(kp, nsteps, progressive, sms, s);
        return tau1 ? run_on<1, true>(kp, nsteps, progressive, sms, s)
                    : run_on<1, false>(kp, nsteps, progressive, sms, s);
    }
    // CTAs per SM that both streaming kernels can keep resident
    static int ctas_per_sm()
    {
        int a, b;
        if constexpr (Store<ST>::DEV) {
            a = occupancy<k_collide_dev<2, true, ST>>();
            b = occupancy<k_macro_dev<2, ST>>();
        } else {
            a = occupancy<k_collide2<true, true>, PART_SMEM>();
            b = occupancy<k_macro2>();
        }
        return a < b ? a : b;
    }
    static cudaError_t sort(const KParams &kp, int sms, cudaStream_t s)
    {
        if (kp.aa) {  // a new visiting order, no moves
            k_sort_rank<<<1, 1024, 0, s>>>(kp);
            return cudaGetLastError();
        }
        // the other arrays first: the population move then leaves the same
        // renumbered populations in both buffers (held cells of the FP32
        // form are never rewritten and are read from either buffer)
        k_sort_rank<<<1, 1024, 0, s>>>(kp);
        k_sort_aux<ST, false><<<sms * 4, THREADS, 0, s>>>(kp);
        k_sort_aux<ST, true><<<sms * 4, THREADS, 0, s>>>(kp);
        k_sort_move<ST><<<sms * 4, THREADS, 0, s>>>(kp);
        k_sort_back<ST><<<sms * 4, THREADS, 0, s>>>(kp);
        k_sort_tables<<<sms * 2, THREADS, 0, s>>>(kp);
        return cudaGetLastError();
    }
    static cudaError_t fused(const KParams &kp, int sms, cudaStream_t s)
    {
        if constexpr (Store<ST>::DEV) {
            return cudaErrorNotSupported;
        } else {
            if (kp.ncomp != 2 || kp.aa || !kp.cflag) return cudaErrorNotSupported;
            if (kp.omega == 1.0f) return launch_fused_grid<k_fused2<true>>(sms, s, kp);
            return launch_fused_grid<k_fused2<false>>(sms, s, kp);
        }
    }
    static const StorageOps *ops()
    {
        static const StorageOps table = {init,    init_finish,  ambient_slot, macro,    activate,    collide,
                                         output,  mass_partial, block_pops,   features, ctas_per_sm, run,
                                         sort,    fused};
        return &table;
    }
};

}  // namespace
}  // namespace lbm
