// Device side of liblbm: the progressive-mesh two-component pseudo-potential
// LBM step (arXiv:1510.03560, Sec. 2 and Sec. 4) for sm_103a.
//
// Layout in HBM (block-major structure of arrays, Sec. 3: SoA for
// coalescing):
//   f[buf][slot][comp][dir][cell]   FP32 populations, two buffers (A-B
//                                   pattern, Sec. 3), cell = x + 8 (y + 8 z)
//   mac[slot][cell]                 float4 (rho0, psi0, rho1, 0) of the step
//   nbits[slot][cell]               bit i: cell x - e_i is solid; bit 19: held
//   uprev[slot][comp][3][cell]      velocity of the previous step, read and
//                                   written only at cells bordering
//                                   unmeshed blocks (criterion, Eq. 13)
// A warp covers four x-rows of one z-plane of a block: every population
// access of a warp touches 4 consecutive 32-byte sectors of one plane.
//
// The step kernels have no block-wide barrier.  A CTA of 256 threads works on
// half a block at a time (grid-stride over half-blocks); every warp fetches
// the slots of the 27 blocks around its block with one lane-parallel load
// and hands them out with shuffles, and reads the per-cell solid bits
// instead of block masks.
//
// One time step is three launches:
//   k_macro    pull streaming + Eqs. 4-5 + Eqs. 6-7 -> mac; criterion of
//              Eq. 13 at cells bordering unmeshed blocks, marking targets
//   k_activate new blocks: slots, ambient equilibrium, their k_macro work
//   k_collide  pull streaming again + forces (Eqs. 8-9, gravity,
//              adhesion) from the neighbours' mac + forced BGK collision
//              (Eqs. 10-12) -> f of the other buffer
#include <climits>
#include <cstdint>

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
constexpr int THREADS = 256;            // threads per CTA of the cell kernels
constexpr int PARTS = CELLS / THREADS;  // CTA work items per block

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

// Neighbour-block index (0..26) of a local coordinate in [-1, 8].
__device__ __forceinline__ int side(int v) { return v < 0 ? 0 : (v > 7 ? 2 : 1); }
__device__ __forceinline__ int nbk(int x, int y, int z) { return side(x) + 3 * side(y) + 9 * side(z); }
__device__ __forceinline__ int lcell(int x, int y, int z)
{
    return (x & 7) | ((y & 7) << 3) | ((z & 7) << 6);
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
    uint32_t mbase;   // first-pass value offset, likewise
};

__device__ __forceinline__ WarpNbr make_nbr(const KParams &kp, int s)
{
    const uint32_t q = s >= 0 ? (uint32_t)s : (uint32_t)kp.amb_slot;
    return WarpNbr{s, __ballot_sync(FULL, s == AMBIENT) & ~(1u << 13), q * (uint32_t)kp.slot_floats,
                   q * (uint32_t)CELLS};
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
__device__ __forceinline__ WarpNbr warp_nbr_of(const KParams &kp, int lane_slot)
{
    return make_nbr(kp, lane_slot);
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
    const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
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

// Pull streaming (Eq. 10, left-hand side) of every component of one cell,
// rest first, then opposite pairs, handing each arriving population to
// sink(a, I, v).  The population moving along e_I comes from x - e_I:
// halfway bounce-back when that cell is solid, the ambient resting
// population when its block is unmeshed, the stored value otherwise; held
// cells keep their own.  With own_ambient the cell's own block is one created
// in this step, still at the ambient state, and is not read back.  All lanes
// must call (shuffles); `live` masks the loads.
template <int NC, class Sink>
__device__ __forceinline__ void pull(const KParams &kp, const WarpNbr &wn, const float *rd,
                                     int own_slot, int c, int lx, int ly, int lz, uint32_t bits,
                                     bool live, bool own_ambient, Sink &&sink)
{
    const uint32_t own =
        (own_ambient ? (uint32_t)kp.amb_slot : (uint32_t)own_slot) * (uint32_t)kp.slot_floats + (uint32_t)c;
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
        for (int c2 = 0; c2 < NC; ++c2) {
            sink.template operator()<I>(c2, v[c2][I]);
        }
    };
    one.template operator()<0>();
    Unroll<0, NPAIR>::run([&]<int P>() {
        one.template operator()<pair_rep(P)>();
        one.template operator()<opp(pair_rep(P))>();
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
// initial velocity as the "previous" one, the cells' solid words.
// in: [slot - slot0][ncomp][4][CELLS] (rho, ux, uy, uz), block-major.
__global__ void __launch_bounds__(CELLS) k_init(KParams kp, const float *in, int slot0, int nslots)
{
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
        for (int a = 0; a < kp.ncomp; ++a) {
            const float *src = in + ((size_t)r * kp.ncomp + a) * 4 * CELLS;
            float rho = src[c], ux = src[CELLS + c], uy = src[2 * CELLS + c],
                  uz = src[3 * CELLS + c];
            if (solid) rho = ux = uy = uz = 0.f;
            const float uu = ux * ux + uy * uy + uz * uz;
            float *d0 = kp.f + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
            float *d1 = d0 + kp.buf_stride;
            Unroll<0, Q>::run([&]<int I>() {
                const float v = feq<I>(wgt(I) * rho, ux, uy, uz, uu);
                d0[I * CELLS] = v;
                d1[I * CELLS] = v;
            });
            if (kp.uprev) {
                float *up = kp.uprev + ((size_t)slot * kp.ncomp + a) * 3 * CELLS + c;
                up[0] = ux;
                up[CELLS] = uy;
                up[2 * CELLS] = uz;
            }
        }
    }
}

// The ambient slot: resting ambient populations in both buffers and the
// ambient first-pass values, read wherever a neighbour block is unmeshed.
__global__ void __launch_bounds__(CELLS) k_ambient_slot(KParams kp)
{
    const int c = threadIdx.x;
    const float psi = psi_of(kp, kp.rho_amb[0]);
    if (c == 0) kp.ctrl->psi_amb = psi;
    for (int a = 0; a < kp.ncomp; ++a) {
        float *d0 = kp.f + (size_t)kp.amb_slot * kp.slot_floats + a * Q * CELLS + c;
        float *d1 = d0 + kp.buf_stride;
        for (int i = 0; i < Q; ++i) {
            d0[i * CELLS] = kp.famb[a][i];
            d1[i * CELLS] = kp.famb[a][i];
        }
    }
    kp.mac[(size_t)kp.amb_slot * CELLS + c] = make_float4(kp.rho_amb[0], psi, kp.rho_amb[1], 0.f);
}

// Streaming + moments of one cell; writes mac (live cells), returns rho and
// the bare velocity.  All lanes must call.
template <int NC>
__device__ __forceinline__ void macro_cell(const KParams &kp, const WarpNbr &wn, const float *rd,
                                           int slot, int c, int lx, int ly, int lz, uint32_t bits,
                                           bool live, bool own_ambient, float rho[2], float u[2][3])
{
    Moments m;
    pull<NC>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, own_ambient,
             [&]<int I>(int a, float v) { m.template add<I>(a, v); });
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        rho[a] = m.rho[a];
        const float inv = 1.f / m.rho[a];
        u[a][0] = m.j[a][0] * inv;
        u[a][1] = m.j[a][1] * inv;
        u[a][2] = m.j[a][2] * inv;
    }
    if (live)
        kp.mac[(size_t)slot * CELLS + c] =
            make_float4(rho[0], psi_of(kp, rho[0]), NC == 2 ? rho[1] : 0.f, 0.f);
}

// Pass 1 of a step: streaming and moments over the meshed blocks; with
// `criterion`, Eq. 13 at fluid cells bordering unmeshed blocks.
template <int NC>
__global__ void __launch_bounds__(THREADS) k_macro(KParams kp, int step, int criterion)
{
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    if (!in_range(kp, n, (long long)kp.capacity + 1, 1)) return;
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    const int lane = threadIdx.x & 31;
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
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
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
        float rho[2], u[2][3];
        macro_cell<NC>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false, rho, u);
        if (criterion) {
            const unsigned front = reach_bits(lx, ly, lz) & wn.amb;
            unsigned tgt = 0;
            if (live && !held && front) {
                float d2max = 0.f;
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                    const float dx = u[a][0] - up[0], dy = u[a][1] - up[CELLS],
                                dz = u[a][2] - up[2 * CELLS];
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
    }
}

// Block creation (Sec. 4.2-4.3): the candidates found by k_macro get slots
// after the meshed ones, start from the ambient resting equilibrium in both
// buffers (R14) and get their streaming and moments of this step computed,
// with every block created in this step seen as ambient.
template <int NC>
__global__ void __launch_bounds__(THREADS) k_activate(KParams kp, int step)
{
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
    }
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    for (int it = blockIdx.x; it < ncand * PARTS; it += gridDim.x) {
        const int k = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
        const int slot = n_old + k;
        const int gid = kp.cand_list[k];
        if (!in_range(kp, gid, (long long)kp.nbx * kp.nby * kp.nbz, 5)) continue;
        if (c == 0) kp.block_of[slot] = gid;
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
        const uint32_t bits = cell_bits(kp, gid, c);
        kp.nbits[(size_t)slot * CELLS + c] = bits;
        const bool live = !(bits & 1u);
        const unsigned fluid = __ballot_sync(FULL, live && !((bits >> HELD_BIT) & 1u));
        if ((threadIdx.x & 31) == 0 && fluid)
            atomicAdd(&ctrl->fluid_active, (unsigned long long)__popc(fluid));
        const WarpNbr wn = warp_nbr(kp, gid, slot, n_old, true);
        float rho[2], u[2][3];
        macro_cell<NC>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, true, rho, u);
    }
}

// Forces on a fluid cell (Eqs. 8-9 as read, gravity, adhesion), from the
// mac values of its 18 neighbours.  A solid neighbour lends the centre's own
// values; an unmeshed one the ambient values.  All lanes must call.
template <int NC>
__device__ __forceinline__ void forces(const KParams &kp, const WarpNbr &wn, int slot, int c,
                                       int lx, int ly, int lz, uint32_t bits, bool live,
                                       const float rho[2], float F[2][3])
{
    const float psi_c = live ? kp.mac[(size_t)slot * CELLS + c].y : 0.f;
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
            psi_n[H] = solid_n ? psi_c : m.y;
            r0_n[H] = solid_n ? r0c : m.x;
            r1_n[H] = solid_n ? r1c : m.z;
            s_n[H] = solid_n ? 1.f : 0.f;
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

// Pass 2 of a step: streaming again, forces, forced BGK collision (Eqs.
// 10-12, R1 sign), store into the other buffer; the velocity is kept for
// the next criterion at cells that border unmeshed blocks.
template <int NC, bool TAU1>
__global__ void __launch_bounds__(THREADS) k_collide(KParams kp, int step)
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
    const int total = n * PARTS;
    int it = blockIdx.x;
    int next_row = it < total ? nbr_row_lane(kp, it / PARTS) : SOLIDBLK;
    uint32_t next_bits =
        it < total ? kp.nbits[(size_t)(it / PARTS) * CELLS + (it % PARTS) * THREADS + threadIdx.x] : 1u;
    for (; it < total; it += gridDim.x) {
        const int slot = it / PARTS;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
        const WarpNbr wn = warp_nbr_of(kp, next_row);
        const uint32_t bits = next_bits;
        const int it2 = it + gridDim.x;
        if (it2 < total) {
            next_row = nbr_row_lane(kp, it2 / PARTS);
            next_bits = kp.nbits[(size_t)(it2 / PARTS) * CELLS + (it2 % PARTS) * THREADS + threadIdx.x];
        }
        const bool live = !(bits & 1u) && !((bits >> HELD_BIT) & 1u);
        if (!__all_sync(FULL, in_range(kp, wn.slot + 2, (long long)kp.capacity + 2, 8))) continue;
        Moments m;
        float fin[TAU1 ? 1 : NC][Q];
        pull<NC>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false, [&]<int I>(int a, float v) {
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
        forces<NC>(kp, wn, slot, c, lx, ly, lz, bits, live, rho, F);
        if (!live) continue;
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
                dst[I * CELLS] = v;
            });
            dst[0] = r - moving;
        }
        if (kp.progressive && (reach_bits(lx, ly, lz) & wn.amb)) {
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

// Macroscopic output of one component for slots [slot0, slot0 + nslots):
// out[slot - slot0][4][CELLS] = rho, ux, uy, uz, velocity u + F / (2 rho)
// at fluid cells (R9), own moments at held cells, zeros at solid cells.
template <int NC>
__global__ void __launch_bounds__(THREADS) k_output(KParams kp, int rdbuf, int comp, int slot0,
                                                    int nslots, float *out)
{
    const float *rd = kp.f + (size_t)rdbuf * kp.buf_stride;
    for (int it = blockIdx.x; it < nslots * PARTS; it += gridDim.x) {
        const int r = it / PARTS;
        const int slot = slot0 + r;
        const int c = (it % PARTS) * THREADS + threadIdx.x;
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
        const WarpNbr wn = warp_nbr_of(kp, nbr_row_lane(kp, slot));
        const uint32_t bits = kp.nbits[(size_t)slot * CELLS + c];
        const bool live = !(bits & 1u);
        const bool held = (bits >> HELD_BIT) & 1u;
        Moments m;
        pull<NC>(kp, wn, rd, slot, c, lx, ly, lz, bits, live, false,
                 [&]<int I>(int a, float v) { m.template add<I>(a, v); });
        float rho[2] = {m.rho[0], m.rho[1]};
        float F[2][3];
        forces<NC>(kp, wn, slot, c, lx, ly, lz, bits, live && !held, rho, F);
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
            }
        }
        float *dst = out + (size_t)r * 4 * CELLS + c;
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q * CELLS] = o[q];
    }
}

// FP64 mass: per-slot partial sums over non-solid cells, then one CTA adds
// the partials in a fixed order.
__global__ void __launch_bounds__(CELLS) k_mass_partial(KParams kp, int rdbuf, int n,
                                                        double *partial)
{
    __shared__ double red[CELLS / 32][2];
    const float *rd = kp.f + (size_t)rdbuf * kp.buf_stride;
    const int c = threadIdx.x;
    for (int slot = blockIdx.x; slot < n; slot += gridDim.x) {
        const bool solid = kp.nbits[(size_t)slot * CELLS + c] & 1u;
        double m[2] = {0.0, 0.0};
        for (int a = 0; a < kp.ncomp; ++a) {
            if (solid) continue;
            const float *src = rd + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += (double)src[i * CELLS];
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

__global__ void __launch_bounds__(1024) k_mass_final(const double *partial, int n, double *out)
{
    __shared__ double red[1024][2];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int i = t; i < n; i += 1024) {
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

}  // namespace

// ---- launch wrappers --------------------------------------------------------

cudaError_t launch_init(const KParams &kp, const float *in_block, int slot0, int nslots, int grid,
                        cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    k_init<<<grid, CELLS, 0, s>>>(kp, in_block, slot0, nslots);
    return cudaGetLastError();
}

cudaError_t launch_ambient_slot(const KParams &kp, cudaStream_t s)
{
    k_ambient_slot<<<1, CELLS, 0, s>>>(kp);
    return cudaGetLastError();
}

// Resident CTAs per SM of a kernel, looked up once per process.
template <class K>
int occupancy(K kernel)
{
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, THREADS, 0) != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        cached = n > 0 ? n : 1;
    }
    return cached;
}

template <class K, class... A>
cudaError_t launch_persistent(K kernel, int sms, cudaStream_t s, A... args)
{
    kernel<<<sms * occupancy(kernel), THREADS, 0, s>>>(args...);
    return cudaGetLastError();
}

cudaError_t launch_macro(const KParams &kp, int step, int criterion, int sms, cudaStream_t s)
{
    if (kp.ncomp == 2) return launch_persistent(k_macro<2>, sms, s, kp, step, criterion);
    return launch_persistent(k_macro<1>, sms, s, kp, step, criterion);
}

cudaError_t launch_activate(const KParams &kp, int step, int sms, cudaStream_t s)
{
    if (kp.ncomp == 2)
        k_activate<2><<<sms, THREADS, 0, s>>>(kp, step);
    else
        k_activate<1><<<sms, THREADS, 0, s>>>(kp, step);
    return cudaGetLastError();
}

cudaError_t launch_collide(const KParams &kp, int step, int sms, cudaStream_t s)
{
    const bool tau1 = kp.omega == 1.0f;
    if (kp.ncomp == 2) {
        if (tau1) return launch_persistent(k_collide<2, true>, sms, s, kp, step);
        return launch_persistent(k_collide<2, false>, sms, s, kp, step);
    }
    if (tau1) return launch_persistent(k_collide<1, true>, sms, s, kp, step);
    return launch_persistent(k_collide<1, false>, sms, s, kp, step);
}

cudaError_t launch_output(const KParams &kp, int rd, int comp, int slot0, int nslots, float *out,
                          int sms, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    if (kp.ncomp == 2) return launch_persistent(k_output<2>, sms, s, kp, rd, comp, slot0, nslots, out);
    return launch_persistent(k_output<1>, sms, s, kp, rd, comp, slot0, nslots, out);
}

cudaError_t launch_mass(const KParams &kp, int rd, int n, double *partial, double *out, int grid,
                        cudaStream_t s)
{
    if (n > 0) {
        k_mass_partial<<<grid, CELLS, 0, s>>>(kp, rd, n, partial);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_mass_final<<<1, 1024, 0, s>>>(partial, n, out);
    return cudaGetLastError();
}

int max_ctas_per_sm_stream_kernels()
{
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_collide<2, true>, THREADS, 0) !=
        cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_macro<2>, THREADS, 0) != cudaSuccess)
        return 1;
    const int n = a < b ? a : b;
    return n > 0 ? n : 1;
}

}  // namespace lbm
