// Device side of liblbm: the progressive-mesh two-component pseudo-potential
// LBM step (arXiv:1510.03560, Sec. 2 and Sec. 4) for sm_103a.
//
// Layout in HBM (block-major structure of arrays, Sec. 3: SoA for
// coalescing):
//   f[buf][slot][comp][dir][cell]   FP32 populations, two buffers (A-B
//                                   pattern, Sec. 3), cell = x + 8 (y + 8 z)
//   mac[slot][3][cell]              rho0, psi0, rho1 of the current step
//   uprev[slot][comp][3][cell]      velocity of the previous step, read and
//                                   written only at cells bordering
//                                   unmeshed blocks (criterion, Eq. 13)
// A warp covers four x-rows of one z-plane of a block, so each population
// access of a warp touches 4 consecutive 32-byte sectors of one plane.
//
// One time step is three launches, each a grid-stride loop of one CTA
// (512 threads, one per cell) per meshed block:
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
// One representative of each opposite pair.
__host__ __device__ constexpr int pair_rep(int p)
{
    return p < 4 ? 1 + 2 * p : 5 + p;  // 1 3 5 7 | 9 10 11 12 13
}
constexpr int NPAIR = 9;

// Neighbour-block index (0..26) of a local coordinate in [-1, 8].
__device__ __forceinline__ int side(int v) { return v < 0 ? 0 : (v > 7 ? 2 : 1); }
__device__ __forceinline__ int nbk(int x, int y, int z) { return side(x) + 3 * side(y) + 9 * side(z); }
__device__ __forceinline__ int lcell(int x, int y, int z)
{
    return (x & 7) | ((y & 7) << 3) | ((z & 7) << 6);
}

// The 3 x 3 x 3 neighbourhood of the block a CTA is working on.
struct Nbr {
    int slot[27];                     // slot, AMBIENT or SOLIDBLK
    uint32_t solid[27][MASK_WORDS];   // solid cells (all set outside the domain)
    uint32_t held[MASK_WORDS];        // held cells of the centre block
    unsigned amb_bits;                // bit k: neighbour k is unmeshed
    unsigned tgt_bits;                // bit k: the criterion fired towards k
};

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
    int bx = gid % kp.nbx, by = (gid / kp.nbx) % kp.nby, bz = gid / (kp.nbx * kp.nby);
    return neighbour_block(kp, bx + k % 3 - 1, by + (k / 3) % 3 - 1, bz + k / 9 - 1);
}

// Fill `nb` for block `gid` held in `own_slot`.  Neighbours whose slot is
// >= slot_limit count as unmeshed (blocks created in the current step,
// seen from the block-creation kernel).  Ends with a barrier.
__device__ void load_neighbourhood(const KParams &kp, int gid, int own_slot, int slot_limit,
                                   Nbr &nb)
{
    const int t = threadIdx.x;
    if (t < 27) {
        int s;
        if (t == 13) {
            s = own_slot;
        } else {
            int nid = neighbour_of(kp, gid, t);
            if (nid < 0) {
                s = SOLIDBLK;
            } else {
                s = kp.slot_of[nid];
                if (s >= slot_limit) s = AMBIENT;
            }
        }
        nb.slot[t] = s;
    }
    for (int w = t; w < 27 * MASK_WORDS; w += blockDim.x) {
        int k = w / MASK_WORDS, word = w % MASK_WORDS;
        int nid = k == 13 ? gid : neighbour_of(kp, gid, k);
        nb.solid[k][word] = nid < 0 ? 0xffffffffu : kp.solid[(size_t)nid * MASK_WORDS + word];
    }
    if (t < MASK_WORDS) nb.held[t] = kp.held[(size_t)gid * MASK_WORDS + t];
    __syncthreads();
    if (t == 0) {
        unsigned bits = 0;
        for (int k = 0; k < 27; ++k)
            if (nb.slot[k] == AMBIENT) bits |= 1u << k;
        nb.amb_bits = bits;
        nb.tgt_bits = 0;
    }
    __syncthreads();
}

__device__ __forceinline__ bool is_solid(const Nbr &nb, int k, int lc)
{
    return (nb.solid[k][lc >> 5] >> (lc & 31)) & 1u;
}

// Neighbour blocks reachable from a cell through the 18 moving velocities.
__device__ __forceinline__ unsigned reach_bits(int lx, int ly, int lz)
{
    unsigned r = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) r |= 1u << nbk(lx + cx(i), ly + cy(i), lz + cz(i));
    return r & ~(1u << 13);
}

// Pull streaming of one component into fin (Eq. 10 left-hand side): the
// population moving along e_i arrives from x - e_i; halfway bounce-back
// when that cell is solid (or outside), the ambient resting population
// when it lies in an unmeshed block.  Held cells keep their own
// populations.
__device__ __forceinline__ void pull(const KParams &kp, const Nbr &nb, const float *rdbuf,
                                     int own_slot, int a, int c, int lx, int ly, int lz,
                                     bool held, float fin[Q])
{
    const float *own = rdbuf + (size_t)own_slot * kp.slot_floats + a * Q * CELLS;
    if (held) {
#pragma unroll
        for (int i = 0; i < Q; ++i) fin[i] = own[i * CELLS + c];
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = lx - cx(i), sy = ly - cy(i), sz = lz - cz(i);
        const int k = nbk(sx, sy, sz);
        const int lc = lcell(sx, sy, sz);
        float v;
        if (is_solid(nb, k, lc)) {
            v = own[opp(i) * CELLS + c];
        } else {
            const int s = nb.slot[k];
            v = s >= 0 ? rdbuf[(size_t)s * kp.slot_floats + a * Q * CELLS + i * CELLS + lc]
                       : kp.famb[a][i];
        }
        fin[i] = v;
    }
}

// Eqs. 4-5: density and momentum (opposite pairs differenced first).
__device__ __forceinline__ void moments(const float fin[Q], float &rho, float j[3])
{
    float r = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) r += fin[i];
    float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        const int i = pair_rep(p);
        const float d = fin[i] - fin[opp(i)];
        if (cx(i) > 0) jx += d; else if (cx(i) < 0) jx -= d;
        if (cy(i) > 0) jy += d; else if (cy(i) < 0) jy -= d;
        if (cz(i) > 0) jz += d; else if (cz(i) < 0) jz -= d;
    }
    rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
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

// ---------------------------------------------------------------------------
// Initial state: equilibrium of the initial fields in both buffers, the
// initial velocity as the "previous" one.  in: [slot - slot0][ncomp][4][CELLS]
// (rho, ux, uy, uz), block-major.
__global__ void __launch_bounds__(CELLS) k_init(KParams kp, const float *in, int slot0, int nslots)
{
    const int c = threadIdx.x;
    for (int r = blockIdx.x; r < nslots; r += gridDim.x) {
        const int slot = slot0 + r;
        const int gid = kp.block_of[slot];
        const bool solid = (kp.solid[(size_t)gid * MASK_WORDS + (c >> 5)] >> (c & 31)) & 1u;
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

__global__ void k_ambient_psi(KParams kp)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) kp.ctrl->psi_amb = psi_of(kp, kp.rho_amb[0]);
}

// Streaming + macroscopics of one cell of a meshed block into mac; returns
// the bare velocities for the criterion.
template <int NC>
__device__ __forceinline__ void macro_cell(const KParams &kp, const Nbr &nb, const float *rd,
                                           int slot, int c, int lx, int ly, int lz, bool held,
                                           float u[2][3])
{
    float rho[2] = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        float fin[Q], j[3];
        pull(kp, nb, rd, slot, a, c, lx, ly, lz, held, fin);
        moments(fin, rho[a], j);
        const float inv = 1.f / rho[a];
        u[a][0] = j[0] * inv;
        u[a][1] = j[1] * inv;
        u[a][2] = j[2] * inv;
    }
    float *m = kp.mac + (size_t)slot * MACS * CELLS + c;
    m[0] = rho[0];
    m[CELLS] = psi_of(kp, rho[0]);
    if (NC == 2) m[2 * CELLS] = rho[1];
}

// Pass 1 of a step: streaming and moments over the meshed blocks; with
// `criterion`, Eq. 13 at fluid cells bordering unmeshed blocks.
template <int NC>
__global__ void __launch_bounds__(CELLS) k_macro(KParams kp, int step, int criterion)
{
    __shared__ Nbr nb;
    Ctrl *ctrl = kp.ctrl;
    if (criterion && ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par];
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    const int c = threadIdx.x, lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
    const unsigned reach = reach_bits(lx, ly, lz);
    for (int slot = blockIdx.x; slot < n; slot += gridDim.x) {
        const int gid = kp.block_of[slot];
        load_neighbourhood(kp, gid, slot, INT_MAX, nb);
        const bool solid = is_solid(nb, 13, c);
        const bool held = (nb.held[c >> 5] >> (c & 31)) & 1u;
        if (!solid) {
            float u[2][3];
            macro_cell<NC>(kp, nb, rd, slot, c, lx, ly, lz, held, u);
            const unsigned front = reach & nb.amb_bits;
            if (criterion && !held && front) {
                float d2max = 0.f;
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    const float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                    const float dx = u[a][0] - up[0], dy = u[a][1] - up[CELLS],
                                dz = u[a][2] - up[2 * CELLS];
                    d2max = fmaxf(d2max, dx * dx + dy * dy + dz * dz);
                }
                if (d2max > kp.S2) atomicOr(&nb.tgt_bits, front);
            }
        }
        __syncthreads();
        if (criterion && threadIdx.x < 27 && ((nb.tgt_bits >> threadIdx.x) & 1u)) {
            const int nid = neighbour_of(kp, gid, threadIdx.x);
            if (atomicCAS(&kp.cand_mark[nid], 0u, 1u) == 0u) {
                const int pos = atomicAdd(&ctrl->ncand[par], 1);
                kp.cand_list[pos] = nid;
            }
        }
        __syncthreads();
    }
}

// Block creation (Sec. 4.2-4.3): the candidates found by k_macro get slots
// after the meshed ones, start from the ambient resting equilibrium in both
// buffers (R14) and get their streaming and moments of this step computed,
// with every block created in this step seen as ambient.
template <int NC>
__global__ void __launch_bounds__(CELLS) k_activate(KParams kp, int step)
{
    __shared__ Nbr nb;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n_old = ctrl->n_active[par];
    const int ncand = ctrl->ncand[par];
    if (n_old + ncand > kp.capacity) {
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
    const int c = threadIdx.x, lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
    for (int k = blockIdx.x; k < ncand; k += gridDim.x) {
        const int slot = n_old + k;
        const int gid = kp.cand_list[k];
        if (threadIdx.x == 0) {
            kp.block_of[slot] = gid;
            kp.slot_of[gid] = slot;
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
        __syncthreads();  // the block's own populations are visible to the CTA
        load_neighbourhood(kp, gid, slot, n_old, nb);
        const bool solid = is_solid(nb, 13, c);
        const bool held = (nb.held[c >> 5] >> (c & 31)) & 1u;
        if (!solid) {
            float u[2][3];
            macro_cell<NC>(kp, nb, rd, slot, c, lx, ly, lz, held, u);
        }
        __syncthreads();
    }
}

// Forces on a fluid cell (Eqs. 8-9 as read, gravity, adhesion), from the
// mac values of its 18 neighbours.  A solid neighbour lends the centre's own
// values; an unmeshed one the ambient values.
template <int NC>
__device__ __forceinline__ void forces(const KParams &kp, const Nbr &nb, int slot, int c, int lx,
                                       int ly, int lz, const float rho[2], float F[2][3])
{
    const float *mc = kp.mac + (size_t)slot * MACS * CELLS;
    const float psi_c = mc[CELLS + c];
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
            if (is_solid(nb, k, lc)) {
                psi_n[H] = psi_c;
                r0_n[H] = r0c;
                r1_n[H] = r1c;
                s_n[H] = 1.f;
            } else {
                const int s = nb.slot[k];
                if (s >= 0) {
                    const float *m = kp.mac + (size_t)s * MACS * CELLS + lc;
                    r0_n[H] = m[0];
                    psi_n[H] = m[CELLS];
                    r1_n[H] = NC == 2 ? m[2 * CELLS] : 0.f;
                } else {
                    r0_n[H] = kp.rho_amb[0];
                    psi_n[H] = kp.psi_amb;
                    r1_n[H] = kp.rho_amb[1];
                }
                s_n[H] = 0.f;
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

// Pass 2 of a step: streaming again, forces, forced BGK collision (Eqs.
// 10-12, R1 sign), store into the other buffer; the velocity is kept for
// the next criterion at cells that border unmeshed blocks.
template <int NC, bool TAU1>
__global__ void __launch_bounds__(CELLS) k_collide(KParams kp, int step)
{
    __shared__ Nbr nb;
    Ctrl *ctrl = kp.ctrl;
    if (ctrl->status) return;
    const int par = step & 1;
    const int n = ctrl->n_active[par ^ 1];
    const float *rd = kp.f + (size_t)par * kp.buf_stride;
    float *wr = kp.f + (size_t)(par ^ 1) * kp.buf_stride;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->cell_updates += (unsigned long long)n * CELLS;
    const int c = threadIdx.x, lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
    const unsigned reach = reach_bits(lx, ly, lz);
    for (int slot = blockIdx.x; slot < n; slot += gridDim.x) {
        const int gid = kp.block_of[slot];
        load_neighbourhood(kp, gid, slot, INT_MAX, nb);
        if (threadIdx.x == 0) {
            int nf = 0;
            for (int w = 0; w < MASK_WORDS; ++w) nf += __popc(~(nb.solid[13][w] | nb.held[w]));
            atomicAdd(&ctrl->fluid_updates, (unsigned long long)nf);
        }
        const bool solid = is_solid(nb, 13, c);
        const bool held = (nb.held[c >> 5] >> (c & 31)) & 1u;
        if (!solid && !held) {
            float fin[NC][Q], rho[2] = {0.f, 0.f}, u[2][3];
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float j[3];
                pull(kp, nb, rd, slot, a, c, lx, ly, lz, false, fin[a]);
                moments(fin[a], rho[a], j);
                const float inv = 1.f / rho[a];
                u[a][0] = j[0] * inv;
                u[a][1] = j[1] * inv;
                u[a][2] = j[2] * inv;
            }
            float F[2][3];
            forces<NC>(kp, nb, slot, c, lx, ly, lz, rho, F);
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                const float inv = 1.f / rho[a];
                const float vx = u[a][0] + F[a][0] * inv, vy = u[a][1] + F[a][1] * inv,
                            vz = u[a][2] + F[a][2] * inv;
                const float vv = vx * vx + vy * vy + vz * vz;
                const float uu = u[a][0] * u[a][0] + u[a][1] * u[a][1] + u[a][2] * u[a][2];
                float *dst = wr + (size_t)slot * kp.slot_floats + a * Q * CELLS + c;
                const float r = rho[a];
                // The 18 moving populations from Eqs. 10-12; the rest
                // population from the mass balance sum_i f_i = rho, which
                // the collision satisfies exactly in real arithmetic.  In
                // FP32 this keeps the mass free of the systematic bias of
                // the rounded weights (fl(1/3) + 6 fl(1/18) + 12 fl(1/36)
                // = 1 + 1.5e-8).
                float moving = 0.f;
                Unroll<1, Q>::run([&]<int I>() {
                    const float wr_ = wgt(I) * r;
                    float v = feq<I>(wr_, vx, vy, vz, vv);
                    if (!TAU1) {
                        const float e0 = feq<I>(wr_, u[a][0], u[a][1], u[a][2], uu);
                        v += (1.f - kp.omega) * (fin[a][I] - e0);
                    }
                    moving += v;
                    dst[I * CELLS] = v;
                });
                dst[0] = r - moving;
            }
            if (kp.progressive && (reach & nb.amb_bits)) {
#pragma unroll
                for (int a = 0; a < NC; ++a) {
                    float *up = kp.uprev + ((size_t)slot * NC + a) * 3 * CELLS + c;
                    up[0] = u[a][0];
                    up[CELLS] = u[a][1];
                    up[2 * CELLS] = u[a][2];
                }
            }
        }
        __syncthreads();
    }
}

// Macroscopic output of one component for slots [slot0, slot0 + nslots):
// out[slot - slot0][4][CELLS] = rho, ux, uy, uz, velocity u + F / (2 rho)
// at fluid cells (R9), own moments at held cells, zeros at solid cells.
template <int NC>
__global__ void __launch_bounds__(CELLS) k_output(KParams kp, int rdbuf, int comp, int slot0,
                                                  int nslots, float *out)
{
    __shared__ Nbr nb;
    const float *rd = kp.f + (size_t)rdbuf * kp.buf_stride;
    const int c = threadIdx.x, lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
    for (int r = blockIdx.x; r < nslots; r += gridDim.x) {
        const int slot = slot0 + r;
        const int gid = kp.block_of[slot];
        load_neighbourhood(kp, gid, slot, INT_MAX, nb);
        const bool solid = is_solid(nb, 13, c);
        const bool held = (nb.held[c >> 5] >> (c & 31)) & 1u;
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        if (!solid) {
            float rho[2] = {0.f, 0.f}, u[2][3];
#pragma unroll
            for (int a = 0; a < NC; ++a) {
                float fin[Q], j[3];
                pull(kp, nb, rd, slot, a, c, lx, ly, lz, held, fin);
                moments(fin, rho[a], j);
                const float inv = 1.f / rho[a];
                u[a][0] = j[0] * inv;
                u[a][1] = j[1] * inv;
                u[a][2] = j[2] * inv;
            }
            const int a = comp;
            o[0] = rho[a];
            o[1] = u[a][0];
            o[2] = u[a][1];
            o[3] = u[a][2];
            if (!held) {
                float F[2][3];
                forces<NC>(kp, nb, slot, c, lx, ly, lz, rho, F);
                const float h = 0.5f / rho[a];
                o[1] += F[a][0] * h;
                o[2] += F[a][1] * h;
                o[3] += F[a][2] * h;
            }
        }
        float *dst = out + (size_t)r * 4 * CELLS + c;
#pragma unroll
        for (int m = 0; m < 4; ++m) dst[m * CELLS] = o[m];
        __syncthreads();
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
        const int gid = kp.block_of[slot];
        const bool solid = (kp.solid[(size_t)gid * MASK_WORDS + (c >> 5)] >> (c & 31)) & 1u;
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
            for (int o = 16; o > 0; o >>= 1) m[a] += __shfl_down_sync(0xffffffffu, m[a], o);
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

cudaError_t launch_ambient_psi(const KParams &kp, cudaStream_t s)
{
    k_ambient_psi<<<1, 32, 0, s>>>(kp);
    return cudaGetLastError();
}

cudaError_t launch_macro(const KParams &kp, int step, int criterion, int grid, cudaStream_t s)
{
    if (kp.ncomp == 2)
        k_macro<2><<<grid, CELLS, 0, s>>>(kp, step, criterion);
    else
        k_macro<1><<<grid, CELLS, 0, s>>>(kp, step, criterion);
    return cudaGetLastError();
}

cudaError_t launch_activate(const KParams &kp, int step, int grid, cudaStream_t s)
{
    if (kp.ncomp == 2)
        k_activate<2><<<grid, CELLS, 0, s>>>(kp, step);
    else
        k_activate<1><<<grid, CELLS, 0, s>>>(kp, step);
    return cudaGetLastError();
}

cudaError_t launch_collide(const KParams &kp, int step, int grid, cudaStream_t s)
{
    const bool tau1 = kp.omega == 1.0f;
    if (kp.ncomp == 2) {
        if (tau1) k_collide<2, true><<<grid, CELLS, 0, s>>>(kp, step);
        else k_collide<2, false><<<grid, CELLS, 0, s>>>(kp, step);
    } else {
        if (tau1) k_collide<1, true><<<grid, CELLS, 0, s>>>(kp, step);
        else k_collide<1, false><<<grid, CELLS, 0, s>>>(kp, step);
    }
    return cudaGetLastError();
}

cudaError_t launch_output(const KParams &kp, int rd, int comp, int slot0, int nslots, float *out,
                          int grid, cudaStream_t s)
{
    if (nslots <= 0) return cudaSuccess;
    if (kp.ncomp == 2)
        k_output<2><<<grid, CELLS, 0, s>>>(kp, rd, comp, slot0, nslots, out);
    else
        k_output<1><<<grid, CELLS, 0, s>>>(kp, rd, comp, slot0, nslots, out);
    return cudaGetLastError();
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
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide<2, true>, CELLS, 0) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace lbm
