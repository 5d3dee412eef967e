// Host runtime of liblbm: the C ABI of include/lbm.h.  It owns the context
// (parameters, block pool, block tables, error state), builds the geometry
// tables, enqueues the kernels of lbm_kernels.cu and moves results to the
// host.  Method: arXiv:1510.03560, Sec. 2 (physics) and Sec. 4 (progressive
// mesh); the per-call references are in include/lbm.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

// The library's velocity order (same table as the kernels).
constexpr int EV[Q][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {1, 1, 0},  {-1, -1, 0},
    {1, -1, 0},  {-1, 1, 0},  {0, 0, 1},  {1, 0, 1},  {-1, 0, 1}, {0, 1, 1},  {0, -1, 1},
    {0, 0, -1},  {-1, 0, -1}, {1, 0, -1}, {0, -1, -1}, {0, 1, -1}};

// The kernels' FP32 weights.
float weight_f(int i)
{
    int n2 = EV[i][0] * EV[i][0] + EV[i][1] * EV[i][1] + EV[i][2] * EV[i][2];
    return n2 == 0 ? 1.0f / 3.0f : (n2 == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

thread_local char g_create_error[512] = "no error";

struct Event {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace

struct lbm_ctx {
    lbm_params p{};
    int device = 0;
    int sms = 1;
    int ctas_per_sm = 1;
    int nbx = 0, nby = 0, nbz = 0;
    int bx = EDGE, by = EDGE, bz = EDGE;  // cells per block along x, y, z
    std::vector<long long> cell_off;     // [CELLS]: grid offset of a block's cell from its origin
    long long nblocks = 0;
    int capacity = 0;
    bool geometry = false;
    long long step = 0;        // completed steps (host view)
    int sticky = LBM_OK;       // error that refuses further steps
    char err[512] = "no error";
    cudaStream_t stream = nullptr;
    KParams kp{};
    // device allocations
    std::vector<void *> allocs;
    std::vector<size_t> alloc_sizes;  // bytes of each entry of allocs
    long long device_bytes = 0;
    int held_rows = 0;                // rows of kp.held_f (A-A streaming)
    double *mass_partial = nullptr;
    double *mass_out = nullptr;
    float *stage = nullptr;    // staging buffer (initial state upload, macro download)
    size_t stage_floats = 0;
    // host copies of the geometry
    std::vector<uint32_t> solid_h, held_h;
    std::vector<int> nonsolid_h;  // non-solid cells per block
    std::vector<int> slot_of_h;   // at set_geometry (static tables)
    float rho_amb[2] = {0.f, 0.f};
    // counters
    long long launches = 0;
    bool profiling = false;
    std::vector<Event> pending;
    std::vector<cudaEvent_t> event_pool;
    double kernel_ms[4] = {0, 0, 0, 0};
    long long kernel_launches[4] = {0, 0, 0, 0};
    // frontier features and the activation proposer
    unsigned *pmark = nullptr;   // [nblocks]
    int *plist = nullptr;        // [nblocks]
    int *pcount = nullptr;       // [1]
    int *pnsnap = nullptr;       // [1]: meshed count taken between two steps
    float *pfeat = nullptr;      // [nblocks][LBM_MLP_IN]
    float *pprob = nullptr;      // [nblocks]
    unsigned *prep = nullptr;    // [nblocks]
    uint32_t *nbits_pre = nullptr;  // [nblocks][CELLS]
    lbm_mlp *mlp = nullptr;
    int period = 0;
    float threshold = 0.5f;
    cudaStream_t side = nullptr;
    cudaEvent_t side_ev = nullptr;
    cudaEvent_t side_done = nullptr;  // end of the side stream's last proposer round
    int sort_period = 64;             // steps between checks for renumbering the slots (0: never)
    // execution mode
    int exec = LBM_EXEC_STREAM;
    cudaStream_t cap = nullptr;        // capture stream of the step graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;   // two steps
    bool graph_fused = false;          // the graph holds fused launches
    // fused step: the collision of step t and pass 1 of step t + 1 in one
    // launch (FP32, two components, A-B, STREAM and GRAPH modes)
    bool fuse = false;
    bool ahead = false;  // pass 1 (with the criterion) of the next step has run
    bool fz_clean = false;  // the arrival counters are set for the next fused launch
    int strip_rows = -1; // slot order: -1 automatic, 0 block order, > 0 strip rows
    // density partials (FP32, two components, A-B; off by default): the
    // collision writes them, the next pass 1 sums them instead of pulling
    bool partials = false;
    bool part_ok = false;     // the last collision wrote them for the current state
    bool graph_part = false;  // the step graph was captured with them
};

namespace {

int fail(lbm_ctx *c, int code, const char *fmt, ...)
{
    char *dst = c ? c->err : g_create_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_OR_FAIL(ctx, call)                                                             \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((ctx), LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

// Keeps the context's device current for the duration of an API call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void *dev_alloc(lbm_ctx *c, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void *ptr = nullptr;
    if (c->p.dev_alloc) {
        ptr = c->p.dev_alloc(bytes, c->p.alloc_user);
    } else if (cudaMallocAsync(&ptr, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) {
        c->allocs.push_back(ptr);
        c->alloc_sizes.push_back(bytes);
        c->device_bytes += (long long)bytes;
    }
    return ptr;
}

void free_all(lbm_ctx *c)
{
    for (void *ptr : c->allocs) {
        if (c->p.dev_free)
            c->p.dev_free(ptr, c->p.alloc_user);
        else
            cudaFreeAsync(ptr, c->stream);
    }
    c->allocs.clear();
    c->alloc_sizes.clear();
    c->device_bytes = 0;
}

// Free one allocation of the context (NULL is accepted).
void release(lbm_ctx *c, void *ptr)
{
    if (!ptr) return;
    for (size_t i = 0; i < c->allocs.size(); ++i)
        if (c->allocs[i] == ptr) {
            c->device_bytes -= (long long)c->alloc_sizes[i];
            c->allocs.erase(c->allocs.begin() + (long)i);
            c->alloc_sizes.erase(c->alloc_sizes.begin() + (long)i);
            if (c->p.dev_free)
                c->p.dev_free(ptr, c->p.alloc_user);
            else
                cudaFreeAsync(ptr, c->stream);
            break;
        }
}

// Grid index of the first cell of block b (its origin); cell lc of the
// block (lc = x + bx (y + by z) in block-local coordinates) is at
// block_origin + cell_off[lc].
long long block_origin(const lbm_ctx *c, long long b)
{
    const long long ix = b % c->nbx, iy = (b / c->nbx) % c->nby, iz = b / ((long long)c->nbx * c->nby);
    return ix * c->bx + (long long)c->p.nx * (iy * c->by + (long long)c->p.ny * (iz * c->bz));
}

// Index of the block shape p asks for in BLOCK_SHAPES ({0, 0, 0}: the
// default), or -1.
int shape_index(const lbm_params *p)
{
    if (p->block[0] == 0 && p->block[1] == 0 && p->block[2] == 0) return 0;
    for (int i = 0; i < NSHAPES; ++i)
        if (p->block[0] == BLOCK_SHAPES[i].x && p->block[1] == BLOCK_SHAPES[i].y &&
            p->block[2] == BLOCK_SHAPES[i].z)
            return i;
    return -1;
}

int validate(const lbm_params *p)
{
    if (!p) return fail(nullptr, LBM_EINVAL, "params is NULL");
    const int si = shape_index(p);
    if (si < 0)
        return fail(nullptr, LBM_EINVAL, "unsupported block shape %dx%dx%d (8x8x8, 16x8x4, 16x4x8, 32x4x4)",
                    p->block[0], p->block[1], p->block[2]);
    const BlockShape sh = BLOCK_SHAPES[si];
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->nx % sh.x || p->ny % sh.y || p->nz % sh.z)
        return fail(nullptr, LBM_EINVAL, "grid %dx%dx%d is not a positive multiple of the %dx%dx%d block",
                    p->nx, p->ny, p->nz, sh.x, sh.y, sh.z);
    if (p->ncomp != 1 && p->ncomp != 2)
        return fail(nullptr, LBM_EINVAL, "ncomp must be 1 or 2, got %d", p->ncomp);
    if (!(p->tau > 0.5) || !std::isfinite(p->tau))
        return fail(nullptr, LBM_EINVAL, "tau must be > 0.5, got %g", p->tau);
    if (!(p->S >= 0.0) || !std::isfinite(p->S))
        return fail(nullptr, LBM_EINVAL, "S must be >= 0, got %g", p->S);
    if (p->max_blocks < 0) return fail(nullptr, LBM_EINVAL, "max_blocks must be >= 0");
    if (p->storage != LBM_STORAGE_FP32 && p->storage != LBM_STORAGE_FP16 &&
        p->storage != LBM_STORAGE_BF16)
        return fail(nullptr, LBM_EINVAL, "unknown storage form %d", p->storage);
    if (p->streaming != LBM_STREAM_AB && p->streaming != LBM_STREAM_AA)
        return fail(nullptr, LBM_EINVAL, "unknown streaming pattern %d", p->streaming);
    if (p->streaming == LBM_STREAM_AA && (p->storage != LBM_STORAGE_FP32 || p->ncomp != 2))
        return fail(nullptr, LBM_EINVAL, "A-A streaming needs the FP32 storage form and two components");
    if (si != 0 && p->storage != LBM_STORAGE_FP32)
        return fail(nullptr, LBM_EINVAL, "block shapes other than 8x8x8 need the FP32 storage form");
    if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr))
        return fail(nullptr, LBM_EINVAL, "dev_alloc and dev_free must be given together");
    for (int a = 0; a < 3; ++a)
        if (p->periodic[a] != 0 && p->periodic[a] != 1)
            return fail(nullptr, LBM_EINVAL, "periodic[%d] must be 0 or 1", a);
    if (p->g_self != 0.0 && (p->pr_b <= 0.0 || p->pr_a <= 0.0 || p->pr_R <= 0.0 ||
                             p->T_over_Tc <= 0.0))
        return fail(nullptr, LBM_EINVAL, "Peng-Robinson a, b, R and T/Tc must be > 0");
    long long nb = (long long)(p->nx / sh.x) * (p->ny / sh.y) * (p->nz / sh.z);
    if (nb > INT32_MAX / 2) return fail(nullptr, LBM_EINVAL, "grid too large");
    return LBM_OK;
}

void fill_physics(lbm_ctx *c)
{
    const lbm_params &p = c->p;
    KParams &k = c->kp;
    k.nbx = c->nbx;
    k.nby = c->nby;
    k.nbz = c->nbz;
    for (int a = 0; a < 3; ++a) k.per[a] = p.periodic[a];
    k.ncomp = p.ncomp;
    k.capacity = c->capacity;
    k.progressive = p.progressive ? 1 : 0;
    k.storage = p.storage;
    k.shape = shape_index(&p);
    k.omega = (float)(1.0 / p.tau);
    k.beta = (float)p.beta;
    k.g_self = (float)p.g_self;
    k.g_cross = (float)p.g_cross;
    for (int a = 0; a < 2; ++a) {
        k.g_ads[a] = (float)p.g_ads[a];
        k.rho_ref[a] = (float)p.rho_ref[a];
    }
    for (int d = 0; d < 3; ++d) k.grav[d] = (float)p.grav[d];
    k.S2 = (float)(p.S * p.S);
    // Peng-Robinson constants (Eq. 7): Tc from a and b, theta(T) the
    // standard alpha function of the acentric factor.
    double Tc = 0.0778 * p.pr_a / (0.45724 * p.pr_b * p.pr_R);
    double T = p.T_over_Tc * Tc;
    double kap = 0.37464 + 1.54226 * p.pr_omega - 0.26992 * p.pr_omega * p.pr_omega;
    double sq = 1.0 + kap * (1.0 - std::sqrt(T / Tc));
    k.pr_b = (float)p.pr_b;
    k.pr_RT = (float)(p.pr_R * T);
    k.pr_atheta = (float)(p.pr_a * sq * sq);
    k.psi_scale = p.g_self != 0.0 ? (float)(2.0 / ((1.0 / 3.0) * p.g_self)) : 0.f;
}

void flush_profile(lbm_ctx *c)
{
    for (Event &e : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            c->kernel_ms[e.kind] += ms;
            c->kernel_launches[e.kind] += 1;
        } else {
            cudaGetLastError();
        }
        c->event_pool.push_back(e.a);
        c->event_pool.push_back(e.b);
    }
    c->pending.clear();
}

cudaEvent_t take_event(lbm_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Launch `fn` (`kernels` kernel launches) with optional timing events
// around it.
template <class F>
cudaError_t timed(lbm_ctx *c, int kind, F &&fn, int kernels = 1)
{
    Event ev{kind, nullptr, nullptr};
    if (c->profiling) {
        ev.a = take_event(c);
        ev.b = take_event(c);
        if (ev.a) cudaEventRecord(ev.a, c->stream);
    }
    cudaError_t e = fn();
    c->launches += kernels;
    if (c->profiling && ev.a && ev.b) {
        cudaEventRecord(ev.b, c->stream);
        c->pending.push_back(ev);
    }
    return e;
}

int persistent_grid(lbm_ctx *c) { return c->sms * c->ctas_per_sm; }

// Bytes of the fused step's arrival counters: two step parities of one int
// per half block of the pool.
size_t cflag_bytes(int capacity) { return (size_t)2 * capacity * 2 * sizeof(int); }

// The fused launch counts arrivals in one parity of its counters and clears
// the other for the next fused launch; any other step breaks that chain, so
// both parities are cleared before the next fused launch.
cudaError_t fused_launch(lbm_ctx *c, cudaStream_t s)
{
    if (!c->fz_clean) {
        cudaError_t e = cudaMemsetAsync(c->kp.cflag, 0, cflag_bytes(c->capacity), s);
        if (e != cudaSuccess) return e;
        c->fz_clean = true;
    }
    return launch_fused(c->kp, c->sms, s);
}

// Strip height of the automatic slot order: about STRIP_BLOCKS blocks per
// strip layer (0: the grid is narrow enough for plain block order).
constexpr int STRIP_BLOCKS = 512;
int auto_strip(int nbx, int nby)
{
    const int rows = std::max(1, STRIP_BLOCKS / std::max(nbx, 1));
    return rows >= nby ? 0 : rows;
}

// The neighbour distance that covers FZ_COVER_PERMIL per mille of the slots
// (as k_sort_tables computes it on the device), from the host's rows.
int lag_distance(const std::vector<int> &rows, int n)
{
    if (n <= 0) return 0;
    std::vector<long long> hist(FZ_BINS, 0);
    for (int s = 0; s < n; ++s) {
        int far = s;
        for (int k = 0; k < NBR_STRIDE; ++k) far = std::max(far, rows[(size_t)s * NBR_STRIDE + k]);
        hist[std::min((far - s) / FZ_BIN, FZ_BINS - 1)] += 1;
    }
    const long long need = ((long long)n * FZ_COVER_PERMIL + 999) / 1000;
    long long cum = 0;
    int b = 0;
    for (; b < FZ_BINS - 1; ++b) {
        cum += hist[b];
        if (cum >= need) break;
    }
    return (b + 1) * FZ_BIN;
}

// Read the device control words after the stream is idle.
int read_ctrl(lbm_ctx *c, Ctrl &out)
{
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&out, c->kp.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                    c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// One round of the activation proposer before step t, on the side stream:
// frontier blocks, their features, the network, the preparation of the
// blocks it selects.  The meshed count is copied on the main stream first,
// so the side stream only reads table rows that are complete.
int enqueue_proposer(lbm_ctx *c, int t)
{
    KParams &k = c->kp;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->pnsnap, &k.ctrl->n_active[t & 1], sizeof(int),
                                    cudaMemcpyDeviceToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaEventRecord(c->side_ev, c->stream));
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->side, c->side_ev, 0));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->pmark, 0, c->nblocks * sizeof(unsigned), c->side));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->pcount, 0, sizeof(int), c->side));
    CUDA_OR_FAIL(c, launch_frontier(k, c->pnsnap, c->pmark, c->plist, c->pcount, c->sms, c->side));
    CUDA_OR_FAIL(c, launch_features(k, t & 1, c->pnsnap, c->plist, c->pcount, c->pfeat, c->sms, c->side));
    CUDA_OR_FAIL(c, mlp_forward_on(c->mlp, c->pfeat, (int)c->nblocks, c->pcount, 1, c->pprob, c->side));
    CUDA_OR_FAIL(c, launch_prepare(k, c->plist, c->pcount, c->pprob, c->threshold, c->prep, c->nbits_pre,
                                   c->sms, c->side));
    CUDA_OR_FAIL(c, cudaEventRecord(c->side_done, c->side));
    c->launches += 4;
    return LBM_OK;
}

void drop_graph(lbm_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

// Whether the steps may run fused.
bool fusable(const lbm_ctx *c)
{
    return c->fuse && c->kp.cflag && (c->exec == LBM_EXEC_STREAM || c->exec == LBM_EXEC_GRAPH);
}

// Whether the collisions write the density partials and pass 1 sums them
// (not with the TMA-staged kernels or the fused step, which keep the pull).
bool part_mode(const lbm_ctx *c) { return c->partials && c->kp.part && !c->kp.staged && !fusable(c); }

// Pass 1 of step t on stream s (criterion in progressive mode), from the
// partials when the last collision wrote them (then two launches with a
// progressive mesh: the warps that border unmeshed blocks pull in the
// second).
cudaError_t macro_on(lbm_ctx *c, int t, cudaStream_t s)
{
    c->kp.part_in = part_mode(c) && c->part_ok ? 1 : 0;
    return launch_macro(c->kp, t, c->p.progressive ? 1 : 0, c->sms, s);
}
int macro_launches(const lbm_ctx *c, bool part_in) { return part_in && c->p.progressive ? 2 : 1; }

cudaError_t collide_on(lbm_ctx *c, int t, cudaStream_t s)
{
    c->kp.part_out = part_mode(c) ? 1 : 0;
    c->part_ok = part_mode(c);
    return launch_collide(c->kp, t, c->sms, s);
}

// The launches of one step on stream s.  Fused: the step's pass 1 has run
// ahead (in the previous step's fused launch), and this step's fused launch
// runs the next step's.
// With the density partials every pass 1 of the graph sums them: it is
// replayed only after a collision wrote them.
cudaError_t launch_step(lbm_ctx *c, cudaStream_t s, bool fused)
{
    cudaError_t e = cudaSuccess;
    if (!fused) {
        c->kp.part_in = part_mode(c) ? 1 : 0;
        e = launch_macro(c->kp, 0, c->p.progressive ? 1 : 0, c->sms, s);
    }
    if (e == cudaSuccess && c->p.progressive) e = launch_activate(c->kp, 0, c->sms, s);
    c->kp.part_out = part_mode(c) ? 1 : 0;
    if (e == cudaSuccess) e = fused ? launch_fused(c->kp, c->sms, s) : launch_collide(c->kp, 0, c->sms, s);
    return e;
}

// Two steps captured as a graph (once; dropped when the parameters change).
int ensure_graph(lbm_ctx *c, bool fused)
{
    if (c->gexec && (c->graph_fused != fused || c->graph_part != part_mode(c))) drop_graph(c);
    if (c->gexec) return LBM_OK;
    if (!c->cap) CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CUDA_OR_FAIL(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_step(c, c->cap, fused);
    if (e == cudaSuccess) e = launch_step(c, c->cap, fused);
    c->graph_fused = fused;
    c->graph_part = part_mode(c);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(c, LBM_ECUDA, "step graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    c->graph = g;
    CUDA_OR_FAIL(c, cudaGraphInstantiate(&c->gexec, g, 0));
    return LBM_OK;
}

// Whether the slots may need renumbering in block order before step t (the
// device decides whether they do; with A-A streaming, which has no idle
// buffer to move them through, only the visiting order changes).
bool sort_point(const lbm_ctx *c, int t)
{
    return c->sort_period > 0 && c->p.progressive && t > 0 && t % c->sort_period == 0;
}

// A step that ends fused leaves the next step's pass 1 done, its candidates
// marked; a renumbering must not meet pending candidates, so the step before
// a renumbering check runs unfused.
bool fuse_step(const lbm_ctx *c, int t) { return fusable(c) && !sort_point(c, t + 1); }

int enqueue_steps(lbm_ctx *c, int nsteps)
{
    int k = 0;
    while (k < nsteps) {
        const int t = (int)(c->step + k);
        if (sort_point(c, t) && !c->ahead) {
            // the side stream reads the tables: let its last round finish
            if (c->mlp) CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->stream, c->side_done, 0));
            CUDA_OR_FAIL(c, timed(c, K_OTHER, [&] { return launch_sort(c->kp, c->sms, c->stream); },
                                  c->kp.aa ? 1 : 6));
        }
        if (c->mlp && t % c->period == 0) {
            int rc = enqueue_proposer(c, t);
            if (rc) return rc;
        }
        // steps up to the next proposer round or renumbering check
        int chunk = nsteps - k;
        if (c->mlp) chunk = std::min(chunk, c->period - t % c->period);
        if (c->sort_period > 0 && c->p.progressive)
            chunk = std::min(chunk, c->sort_period - t % c->sort_period);
        if (c->exec == LBM_EXEC_PERSISTENT) {
            // (its first pass 1 repeats one that ran ahead, with the same
            // result: the criterion's marks are idempotent)
            c->kp.part_in = part_mode(c) && c->part_ok ? 1 : 0;
            c->kp.part_out = part_mode(c) ? 1 : 0;
            c->part_ok = part_mode(c);
            CUDA_OR_FAIL(c, timed(c, K_OTHER, [&] {
                             return launch_run(c->kp, chunk, c->p.progressive ? 1 : 0, c->sms, c->stream);
                         }));
            c->ahead = false;
            c->fz_clean = false;
            k += chunk;
            continue;
        }
        if (c->exec == LBM_EXEC_GRAPH) {
            const bool fz = fusable(c);
            // fused: the last step before a renumbering check runs unfused
            const int ng = fz && sort_point(c, t + chunk) ? chunk - 1 : chunk;
            // (the graph's passes 1 sum the density partials: a plain step
            // writes them first)
            if (ng >= 2 && (!part_mode(c) || c->part_ok)) {
                if (fz && !c->ahead) {
                    CUDA_OR_FAIL(c, timed(c, K_MACRO, [&] { return macro_on(c, t, c->stream); }));
                    c->ahead = true;
                }
                int rc = ensure_graph(c, fz);
                if (rc) return rc;
                if (fz && !c->fz_clean) {
                    CUDA_OR_FAIL(c, cudaMemsetAsync(c->kp.cflag, 0, cflag_bytes(c->capacity), c->stream));
                    c->fz_clean = true;
                }
                const int per_step =
                    (fz ? 1 : 1 + macro_launches(c, part_mode(c))) + (c->p.progressive ? 1 : 0);
                for (int p = 0; p < ng / 2; ++p)
                    CUDA_OR_FAIL(c, timed(c, K_OTHER, [&] { return cudaGraphLaunch(c->gexec, c->stream); },
                                          2 * per_step));
                c->ahead = fz;
                if (!fz) c->fz_clean = false;
                c->part_ok = part_mode(c);
                k += 2 * (ng / 2);
                continue;
            }
        }
        if (!c->ahead)
            CUDA_OR_FAIL(c, timed(c, K_MACRO, [&] { return macro_on(c, t, c->stream); },
                                  macro_launches(c, part_mode(c) && c->part_ok)));
        if (c->p.progressive)
            CUDA_OR_FAIL(c, timed(c, K_ACTIVATE,
                                  [&] { return launch_activate(c->kp, t, c->sms, c->stream); }));
        if (fuse_step(c, t)) {
            CUDA_OR_FAIL(c, timed(c, K_COLLIDE, [&] { return fused_launch(c, c->stream); }));
            c->ahead = true;
            c->part_ok = false;
        } else {
            CUDA_OR_FAIL(c, timed(c, K_COLLIDE, [&] { return collide_on(c, t, c->stream); }));
            c->ahead = false;
            c->fz_clean = false;
        }
        k += 1;
    }
    c->step += nsteps;
    return LBM_OK;
}

int finish(lbm_ctx *c)
{
    if (c->side) CUDA_OR_FAIL(c, cudaStreamSynchronize(c->side));
    Ctrl ctrl;
    int rc = read_ctrl(c, ctrl);
    if (rc) return rc;
    if (c->profiling) flush_profile(c);
    if (ctrl.check_site != 0) {
        c->sticky = LBM_ECUDA;
        return fail(c, LBM_ECUDA, "device index check %d failed (value %lld)", ctrl.check_site,
                    ctrl.check_value);
    }
    if (ctrl.status != 0) {
        c->step = ctrl.fail_step;
        c->sticky = ctrl.status;
        if (ctrl.status == LBM_ENOMEM)
            return fail(c, LBM_ENOMEM,
                        "block pool full at step %d: %d meshed + %d new blocks > capacity %d",
                        ctrl.fail_step, ctrl.n_active[ctrl.fail_step & 1],
                        ctrl.ncand[ctrl.fail_step & 1], c->capacity);
        if (ctrl.status == LBM_ETIMEOUT) {
            c->step = ctrl.step;
            return fail(c, LBM_ETIMEOUT, "a grid barrier wait timed out after step %d", ctrl.step);
        }
        return fail(c, ctrl.status, "device error %d at step %d", ctrl.status, ctrl.fail_step);
    }
    return LBM_OK;
}

int active_count(lbm_ctx *c, int *n)
{
    Ctrl ctrl;
    int rc = read_ctrl(c, ctrl);
    if (rc) return rc;
    *n = ctrl.n_active[c->step & 1];
    return LBM_OK;
}

}  // namespace

void lbm::set_global_error(const char *msg) { snprintf(g_create_error, sizeof g_create_error, "%s", msg); }

extern "C" {

int lbm_create(const lbm_params *p, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->p = *p;
    c->stream = (cudaStream_t)p->stream;
    const BlockShape sh = BLOCK_SHAPES[shape_index(p)];
    c->bx = sh.x;
    c->by = sh.y;
    c->bz = sh.z;
    c->nbx = p->nx / sh.x;
    c->nby = p->ny / sh.y;
    c->nbz = p->nz / sh.z;
    c->cell_off.resize(CELLS);
    for (int lc = 0; lc < CELLS; ++lc)
        c->cell_off[lc] = lc % sh.x + (long long)p->nx * ((lc / sh.x) % sh.y + (long long)p->ny * (lc / (sh.x * sh.y)));
    c->nblocks = (long long)c->nbx * c->nby * c->nbz;
    long long cap = p->max_blocks > 0 ? std::min<long long>(p->max_blocks, c->nblocks) : c->nblocks;
    c->capacity = (int)cap;
    auto bail = [&](int code) {
        snprintf(g_create_error, sizeof g_create_error, "%s", c->err);
        free_all(c);
        delete c;
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        fail(c, LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(LBM_ECUDA);
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    c->ctas_per_sm = max_ctas_per_sm_stream_kernels(p->storage);
    fill_physics(c);
    c->kp.barrier_spins = 1ll << 24;  // about a second of polling

    const bool dev16 = p->storage != LBM_STORAGE_FP32;
    const size_t slot_floats = (size_t)(dev16 ? 1 : p->ncomp) * Q * CELLS;
    KParams &k = c->kp;
    k.slot_floats = (int)slot_floats;
    k.amb_slot = c->capacity;
    const size_t one_buf = slot_floats * (size_t)(c->capacity + 1);
    if (one_buf >= (1ull << 32)) {
        fail(c, LBM_EINVAL, "block pool of %d blocks too large for 32-bit offsets", c->capacity);
        return bail(LBM_EINVAL);
    }
    // A-A streaming: one array, addressed by both parities (stride 0)
    const bool aa = p->streaming == LBM_STREAM_AA;
    k.aa = aa ? 1 : 0;
    k.buf_stride = aa ? 0 : one_buf;
    const bool fz = !dev16 && !aa && p->ncomp == 2;
    k.strip = auto_strip(c->nbx, c->nby);
    struct Want {
        void **dst;
        size_t bytes;
    } want[] = {
        {(void **)&k.f, dev16 ? 0 : (aa ? 1 : 2) * one_buf * sizeof(float)},
        {(void **)&k.h, dev16 ? 2 * one_buf * sizeof(uint32_t) : 0},
        {(void **)&k.held_rank, aa ? (size_t)c->nblocks * sizeof(int) : 0},
        {(void **)&k.order, aa ? (size_t)c->capacity * sizeof(int) : 0},
        {(void **)&k.mac, (dev16 ? 2 : 1) * (size_t)(c->capacity + 1) * CELLS * sizeof(float4)},
        {(void **)&k.nbits, (size_t)c->capacity * CELLS * sizeof(uint32_t)},
        {(void **)&k.nbr, (size_t)c->capacity * NBR_STRIDE * sizeof(int)},
        {(void **)&k.uprev, p->progressive || dev16 ? (size_t)c->capacity * p->ncomp * 3 * CELLS * sizeof(float) : 0},
        {(void **)&k.slot_of, (size_t)c->nblocks * sizeof(int)},
        {(void **)&k.block_of, (size_t)c->capacity * sizeof(int)},
        {(void **)&k.solid, (size_t)c->nblocks * MASK_WORDS * sizeof(uint32_t)},
        {(void **)&k.held, (size_t)c->nblocks * MASK_WORDS * sizeof(uint32_t)},
        {(void **)&k.cand_list, (size_t)c->nblocks * sizeof(int)},
        {(void **)&k.cand_mark, (size_t)c->nblocks * sizeof(unsigned)},
        {(void **)&k.act_step, (size_t)c->nblocks * sizeof(int)},
        {(void **)&k.ctrl, sizeof(Ctrl)},
        {(void **)&c->mass_partial, (size_t)c->capacity * 2 * sizeof(double)},
        {(void **)&c->mass_out, 2 * sizeof(double)},
        // fused step (FP32, two components, A-B)
        {(void **)&k.cflag, fz ? cflag_bytes(c->capacity) : 0},
        {(void **)&k.fz_hist, fz ? (size_t)FZ_BINS * sizeof(int) : 0},
        // density partials (likewise)
        {(void **)&k.part, fz ? (size_t)c->capacity * CELLS * sizeof(float2) : 0},
        {(void **)&k.recv, fz ? (size_t)c->capacity * 2 * recv_entries(sh.x, sh.y, sh.z) * sizeof(float2) : 0},
    };
    for (auto &w : want) {
        if (w.bytes == 0) {
            *w.dst = nullptr;
            continue;
        }
        *w.dst = dev_alloc(c, w.bytes);
        if (!*w.dst) {
            fail(c, LBM_ENOMEM, "device allocation of %zu bytes failed", w.bytes);
            return bail(LBM_ENOMEM);
        }
    }
    k.mac_stride = dev16 ? (size_t)(c->capacity + 1) * CELLS : 0;
    // staging: up to 2048 blocks of [ncomp][4][CELLS] floats at a time, and
    // at least one block's populations
    c->stage_floats = (size_t)std::min(c->capacity, 2048) * p->ncomp * 4 * CELLS;
    c->stage_floats = std::max(c->stage_floats, (size_t)p->ncomp * Q * CELLS);
    c->stage = (float *)dev_alloc(c, c->stage_floats * sizeof(float));
    if (!c->stage) {
        fail(c, LBM_ENOMEM, "staging allocation failed");
        return bail(LBM_ENOMEM);
    }
    if (fz && (cudaMemsetAsync(k.cflag, 0, cflag_bytes(c->capacity), c->stream) != cudaSuccess ||
               cudaMemsetAsync(k.fz_hist, 0, (size_t)FZ_BINS * sizeof(int), c->stream) != cudaSuccess)) {
        fail(c, LBM_ECUDA, "memset failed");
        return bail(LBM_ECUDA);
    }
    if (cudaMemsetAsync(k.ctrl, 0, sizeof(Ctrl), c->stream) != cudaSuccess) {
        fail(c, LBM_ECUDA, "memset failed");
        return bail(LBM_ECUDA);
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx *c)
{
    if (!c) return LBM_OK;
    DeviceGuard g(c->device);
    if (c->side) cudaStreamSynchronize(c->side);
    cudaStreamSynchronize(c->stream);
    flush_profile(c);
    free_all(c);
    if (c->side_ev) cudaEventDestroy(c->side_ev);
    if (c->side_done) cudaEventDestroy(c->side_done);
    if (c->side) cudaStreamDestroy(c->side);
    drop_graph(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return LBM_OK;
}

int lbm_set_geometry(lbm_ctx *c, const uint8_t *cell_type, const float *rho_init,
                     const float *u_init, const float *rho_amb)
{
    if (!c) return LBM_EINVAL;
    if (!cell_type || !rho_init || !rho_amb)
        return fail(c, LBM_EINVAL, "cell_type, rho_init and rho_amb are required");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, LBM_ECUDA, "cannot select device %d", c->device);
    if (c->side) CUDA_OR_FAIL(c, cudaStreamSynchronize(c->side));
    drop_graph(c);
    const lbm_params &p = c->p;
    const long long ncell = (long long)p.nx * p.ny * p.nz;
    const int nc = p.ncomp;
    for (long long i = 0; i < ncell; ++i)
        if (cell_type[i] > 2) return fail(c, LBM_EINVAL, "cell_type[%lld] = %d", i, cell_type[i]);
    for (int a = 0; a < nc; ++a) {
        if (!std::isfinite(rho_amb[a]) || !(rho_amb[a] > 0.f))
            return fail(c, LBM_EINVAL, "rho_amb[%d] must be a positive number", a);
        c->rho_amb[a] = rho_amb[a];
    }

    // per-block masks, ambient test, initial active set
    const long long nb = c->nblocks;
    c->solid_h.assign(nb * MASK_WORDS, 0u);
    c->held_h.assign(nb * MASK_WORDS, 0u);
    c->nonsolid_h.assign(nb, 0);
    std::vector<char> differs(nb, 0);
    // block index and block-local part of each coordinate, per axis
    std::vector<int> qx(p.nx), rx(p.nx), qy(p.ny), ry(p.ny), qz(p.nz), rz(p.nz);
    for (int x = 0; x < p.nx; ++x) qx[x] = x / c->bx, rx[x] = x % c->bx;
    for (int y = 0; y < p.ny; ++y) qy[y] = y / c->by, ry[y] = (y % c->by) * c->bx;
    for (int z = 0; z < p.nz; ++z) qz[z] = z / c->bz, rz[z] = (z % c->bz) * c->bx * c->by;
    for (int z = 0; z < p.nz; ++z)
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                const long long i = x + (long long)p.nx * (y + (long long)p.ny * z);
                const long long b = qx[x] + c->nbx * ((long long)qy[y] + (long long)c->nby * qz[z]);
                const int lc = rx[x] + ry[y] + rz[z];
                if (cell_type[i] == LBM_CELL_SOLID) {
                    c->solid_h[b * MASK_WORDS + (lc >> 5)] |= 1u << (lc & 31);
                    continue;
                }
                if (cell_type[i] == LBM_CELL_HELD) c->held_h[b * MASK_WORDS + (lc >> 5)] |= 1u << (lc & 31);
                c->nonsolid_h[b] += 1;
                for (int a = 0; a < nc; ++a) {
                    float r = rho_init[a * ncell + i];
                    if (!std::isfinite(r) || !(r > 0.f))
                        return fail(c, LBM_EINVAL, "rho_init[%d][%lld] must be a positive number", a, i);
                    bool d = r != rho_amb[a];
                    if (u_init)
                        for (int k = 0; k < 3; ++k) d = d || u_init[(a * 3 + k) * ncell + i] != 0.f;
                    if (d) differs[b] = 1;
                }
            }
    std::vector<int> slot_of(nb, AMBIENT), block_of;
    for (long long b = 0; b < nb; ++b) {
        if (c->nonsolid_h[b] == 0) {
            slot_of[b] = SOLIDBLK;
            for (int w = 0; w < MASK_WORDS; ++w) c->solid_h[b * MASK_WORDS + w] = 0xffffffffu;
        }
    }
    // initial slots in the slot order (block order, or strips of block rows)
    c->kp.strip = c->strip_rows < 0 ? auto_strip(c->nbx, c->nby) : (c->strip_rows >= c->nby ? 0 : c->strip_rows);
    for (long long r = 0; r < nb; ++r) {
        const long long b = strip_block((int)r, c->nbx, c->nby, c->nbz, c->kp.strip);
        if (c->nonsolid_h[b] > 0 && (!p.progressive || differs[b])) {
            slot_of[b] = (int)block_of.size();
            block_of.push_back((int)b);
        }
    }
    const int n0 = (int)block_of.size();
    if (n0 > c->capacity)
        return fail(c, LBM_ENOMEM, "%d initial blocks exceed the pool capacity %d", n0, c->capacity);

    KParams &k = c->kp;
    for (int a = 0; a < 2; ++a) {
        k.rho_amb[a] = a < nc ? rho_amb[a] : 0.f;
        for (int i = 0; i < Q; ++i) k.famb[a][i] = weight_f(i) * k.rho_amb[a];
    }
    // neighbour-slot rows of the initial slots (k = dx+1 + 3(dy+1) + 9(dz+1))
    std::vector<int> nbr_rows((size_t)std::max(n0, 1) * NBR_STRIDE, SOLIDBLK);
    for (int sl = 0; sl < n0; ++sl) {
        const int b = block_of[sl];
        const int bx = b % c->nbx, by = (b / c->nbx) % c->nby, bz = b / (c->nbx * c->nby);
        for (int kk = 0; kk < 27; ++kk) {
            int q[3] = {bx + kk % 3 - 1, by + (kk / 3) % 3 - 1, bz + kk / 9 - 1};
            const int nq[3] = {c->nbx, c->nby, c->nbz};
            bool outside = false;
            for (int a = 0; a < 3; ++a) {
                if (q[a] < 0 || q[a] >= nq[a]) {
                    if (!p.periodic[a]) outside = true;
                    q[a] = (q[a] + nq[a]) % nq[a];
                }
            }
            int v = SOLIDBLK;
            if (kk == 13) v = sl;
            else if (!outside) v = slot_of[q[0] + c->nbx * ((long long)q[1] + (long long)c->nby * q[2])];
            nbr_rows[(size_t)sl * NBR_STRIDE + kk] = v;
        }
    }
    cudaStream_t s = c->stream;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(k.slot_of, slot_of.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
    if (n0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(k.nbr, nbr_rows.data(), (size_t)n0 * NBR_STRIDE * sizeof(int),
                                        cudaMemcpyHostToDevice, s));
    if (n0)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(k.block_of, block_of.data(), n0 * sizeof(int), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync((void *)k.solid, c->solid_h.data(), nb * MASK_WORDS * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync((void *)k.held, c->held_h.data(), nb * MASK_WORDS * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    if (k.aa) {
        // A-A: a row of constant populations for every block holding held cells
        std::vector<int> rank(nb, -1);
        int nheld = 0;
        for (long long b = 0; b < nb; ++b)
            for (int w = 0; w < MASK_WORDS; ++w)
                if (c->held_h[b * MASK_WORDS + w]) {
                    rank[b] = nheld++;
                    break;
                }
        if (nheld > c->held_rows) {
            CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
            release(c, k.held_f);
            k.held_f = (float *)dev_alloc(c, (size_t)nheld * k.slot_floats * sizeof(float));
            if (!k.held_f) {
                c->held_rows = 0;
                return fail(c, LBM_ENOMEM, "device allocation of the held-cell table failed");
            }
            c->held_rows = nheld;
        }
        CUDA_OR_FAIL(c, cudaMemcpyAsync((void *)k.held_rank, rank.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    }
    CUDA_OR_FAIL(c, cudaMemsetAsync(k.cand_mark, 0, nb * sizeof(unsigned), s));
    c->ahead = false;
    c->fz_clean = false;
    c->part_ok = false;
    {
        std::vector<int> act(nb, -1);
        for (int sl = 0; sl < n0; ++sl) act[block_of[sl]] = 0;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(k.act_step, act.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    }
    if (c->prep) CUDA_OR_FAIL(c, cudaMemsetAsync(c->prep, 0, nb * sizeof(unsigned), s));
    Ctrl ctrl{};
    ctrl.n_active[0] = ctrl.n_active[1] = n0;
    ctrl.fz_dist = lag_distance(nbr_rows, n0);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(k.ctrl, &ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    if (k.mac_stride)
        CUDA_OR_FAIL(c, cudaMemsetAsync(k.mac, 0, 2 * k.mac_stride * sizeof(float4), s));
    CUDA_OR_FAIL(c, launch_ambient_slot(k, s));
    float psi_amb = 0.f;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&psi_amb, &k.ctrl->psi_amb, sizeof(float), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    k.psi_amb = psi_amb;

    // initial populations, staged block-major in chunks
    const int per_chunk = (int)(c->stage_floats / ((size_t)nc * 4 * CELLS));
    std::vector<float> host((size_t)per_chunk * nc * 4 * CELLS);
    for (int s0 = 0; s0 < n0; s0 += per_chunk) {
        const int m = std::min(per_chunk, n0 - s0);
        for (int r = 0; r < m; ++r) {
            const long long o = block_origin(c, block_of[s0 + r]);
            for (int a = 0; a < nc; ++a) {
                float *dst = host.data() + ((size_t)r * nc + a) * 4 * CELLS;
                for (int lc = 0; lc < CELLS; ++lc) {
                    const long long i = o + c->cell_off[lc];
                    dst[lc] = rho_init[a * ncell + i];
                    for (int d = 0; d < 3; ++d)
                        dst[(d + 1) * CELLS + lc] = u_init ? u_init[(a * 3 + d) * ncell + i] : 0.f;
                }
            }
        }
        CUDA_OR_FAIL(c, cudaMemcpyAsync(c->stage, host.data(), (size_t)m * nc * 4 * CELLS * sizeof(float),
                                        cudaMemcpyHostToDevice, s));
        CUDA_OR_FAIL(c, launch_init(k, c->stage, s0, m, std::min(m, persistent_grid(c)), s));
        c->launches += 1;
        CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    }
    CUDA_OR_FAIL(c, launch_init_finish(k, n0, c->sms, s));
    c->launches += k.mac_stride && n0 ? 1 : 0;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    c->slot_of_h = slot_of;
    c->step = 0;
    c->sticky = LBM_OK;
    c->geometry = true;
    return LBM_OK;
}

int lbm_step_async(lbm_ctx *c, int nsteps)
{
    if (!c) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    if (c->sticky) return fail(c, LBM_ESTATE, "stepping refused after an earlier error (%d)", c->sticky);
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps must be >= 0");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(c, LBM_ECUDA, "cannot select device %d", c->device);
    return enqueue_steps(c, nsteps);
}

int lbm_sync(lbm_ctx *c)
{
    if (!c) return LBM_EINVAL;
    DeviceGuard g(c->device);
    return finish(c);
}

int lbm_step(lbm_ctx *c, int nsteps)
{
    int rc = lbm_step_async(c, nsteps);
    if (rc) return rc;
    return lbm_sync(c);
}

int lbm_get_macro(lbm_ctx *c, int comp, float *rho, float *ux, float *uy, float *uz)
{
    if (!c) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    if (comp < 0 || comp >= c->p.ncomp) return fail(c, LBM_EINVAL, "comp %d out of range", comp);
    DeviceGuard g(c->device);
    const lbm_params &p = c->p;
    const long long ncell = (long long)p.nx * p.ny * p.nz;
    float *outs[4] = {rho, ux, uy, uz};
    // unmeshed and solid cells first
    for (long long b = 0; b < c->nblocks; ++b) {
        const long long o = block_origin(c, b);
        for (int lc = 0; lc < CELLS; ++lc) {
            const long long i = o + c->cell_off[lc];
            const bool sol = (c->solid_h[b * MASK_WORDS + (lc >> 5)] >> (lc & 31)) & 1u;
            if (rho) rho[i] = sol ? 0.f : c->rho_amb[comp];
            for (int m = 1; m < 4; ++m)
                if (outs[m]) outs[m][i] = 0.f;
        }
    }
    (void)ncell;
    Ctrl ctrl;
    int rc = read_ctrl(c, ctrl);
    if (rc) return rc;
    const int n = ctrl.n_active[c->step & 1];
    if (n == 0) return LBM_OK;
    std::vector<int> block_of(n);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(block_of.data(), c->kp.block_of, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    const int rd = (int)(c->step & 1);
    c->kp.part_in = part_mode(c) && c->part_ok ? 1 : 0;
    CUDA_OR_FAIL(c, launch_macro(c->kp, (int)c->step, 0, c->sms, c->stream));
    c->launches += macro_launches(c, c->kp.part_in != 0);
    const int per_chunk = (int)(c->stage_floats / (4 * CELLS));
    std::vector<float> host((size_t)per_chunk * 4 * CELLS);
    for (int s0 = 0; s0 < n; s0 += per_chunk) {
        const int m = std::min(per_chunk, n - s0);
        CUDA_OR_FAIL(c, launch_output(c->kp, rd, comp, s0, m, c->stage, c->sms, c->stream));
        c->launches += 1;
        CUDA_OR_FAIL(c, cudaMemcpyAsync(host.data(), c->stage, (size_t)m * 4 * CELLS * sizeof(float),
                                        cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
        for (int r = 0; r < m; ++r) {
            const long long o = block_origin(c, block_of[s0 + r]);
            for (int lc = 0; lc < CELLS; ++lc) {
                const long long i = o + c->cell_off[lc];
                for (int q = 0; q < 4; ++q)
                    if (outs[q]) outs[q][i] = host[((size_t)r * 4 + q) * CELLS + lc];
            }
        }
    }
    return LBM_OK;
}

int lbm_active_blocks(lbm_ctx *c, int32_t *ids, long long cap, long long *n)
{
    if (!c || !n) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    if (cap > 0 && !ids) return fail(c, LBM_EINVAL, "ids is NULL");
    DeviceGuard g(c->device);
    int na = 0;
    int rc = active_count(c, &na);
    if (rc) return rc;
    std::vector<int32_t> all(na);
    if (na) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(all.data(), c->kp.block_of, na * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    }
    std::sort(all.begin(), all.end());
    *n = na;
    for (long long i = 0; i < std::min<long long>(cap, na); ++i) ids[i] = all[i];
    return LBM_OK;
}

int lbm_mass(lbm_ctx *c, double *mass)
{
    if (!c || !mass) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    DeviceGuard g(c->device);
    int na = 0;
    int rc = active_count(c, &na);
    if (rc) return rc;
    std::vector<int32_t> act(na);
    if (na)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(act.data(), c->kp.block_of, na * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    const int rd = (int)(c->step & 1);
    CUDA_OR_FAIL(c, launch_mass(c->kp, rd, na, c->mass_partial, c->mass_out,
                                std::max(1, std::min(na, persistent_grid(c))), c->stream));
    c->launches += na > 0 ? 2 : 1;
    double dev[2] = {0, 0};
    CUDA_OR_FAIL(c, cudaMemcpyAsync(dev, c->mass_out, sizeof dev, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    std::vector<char> meshed(c->nblocks, 0);
    for (int b : act) meshed[b] = 1;
    long long amb_cells = 0;
    for (long long b = 0; b < c->nblocks; ++b)
        if (!meshed[b]) amb_cells += c->nonsolid_h[b];
    for (int a = 0; a < c->p.ncomp; ++a) {
        double per = 0.0;
        for (int i = 0; i < Q; ++i) per += (double)c->kp.famb[a][i];
        mass[a] = dev[a] + per * (double)amb_cells;
    }
    return LBM_OK;
}

int lbm_get_block_populations(lbm_ctx *c, int32_t block_id, float *out)
{
    if (!c || !out) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    if (block_id < 0 || block_id >= c->nblocks) return fail(c, LBM_EINVAL, "block %d out of range", block_id);
    DeviceGuard g(c->device);
    int slot = -1, na = 0;
    int rc = active_count(c, &na);
    if (rc) return rc;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&slot, c->kp.slot_of + block_id, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    // (a candidate already marked for the next step holds a slot >= na)
    if (slot < 0 || slot >= na) return fail(c, LBM_EINVAL, "block %d is not meshed", block_id);
    const int rd = (int)(c->step & 1);
    const bool gather = !c->kp.f || c->kp.aa;  // 16-bit forms decode, A-A gathers
    const float *src = !gather ? c->kp.f + (size_t)rd * c->kp.buf_stride + (size_t)slot * c->kp.slot_floats
                               : c->stage;
    if (gather) {
        CUDA_OR_FAIL(c, launch_block_pops(c->kp, rd, slot, c->stage, c->stream));
        c->launches += 1;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(out, src, (size_t)c->p.ncomp * Q * CELLS * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_velocities(int32_t *e)
{
    if (!e) return LBM_EINVAL;
    for (int i = 0; i < Q; ++i)
        for (int d = 0; d < 3; ++d) e[3 * i + d] = EV[i][d];
    return LBM_OK;
}

int lbm_set_profiling(lbm_ctx *c, int on)
{
    if (!c) return LBM_EINVAL;
    c->profiling = on != 0;
    return LBM_OK;
}

int lbm_get_stats(lbm_ctx *c, lbm_stats *out)
{
    if (!c || !out) return LBM_EINVAL;
    DeviceGuard g(c->device);
    std::memset(out, 0, sizeof *out);
    out->capacity = c->capacity;
    out->total_blocks = c->nblocks;
    out->launches = c->launches;
    out->device_bytes = c->device_bytes;
    out->steps = c->step;
    if (c->geometry) {
        Ctrl ctrl;
        int rc = read_ctrl(c, ctrl);
        if (rc) return rc;
        flush_profile(c);
        out->active_blocks = ctrl.n_active[c->step & 1];
        out->cell_updates = (long long)ctrl.cell_updates;
        out->fluid_updates = (long long)ctrl.fluid_updates;
        out->created_blocks = (long long)ctrl.created;
        out->prepared_blocks = (long long)ctrl.prepared;
        out->prepared_hits = (long long)ctrl.prepared_hits;
        out->slot_sorts = (long long)ctrl.sorts;
        out->fused_deferred = (long long)ctrl.fz_deferred;
        out->fused_waited = (long long)ctrl.fz_waited;
        out->fused_lag_distance = ctrl.fz_dist;
        long long ns = 0;
        for (int v : c->nonsolid_h) ns += v > 0;
        out->nonsolid_blocks = ns;
    }
    for (int k = 0; k < 4; ++k) {
        out->kernel_ms[k] = c->kernel_ms[k];
        out->kernel_launches[k] = c->kernel_launches[k];
    }
    return LBM_OK;
}

// Buffers of the frontier features (and of the proposer), on first use.
static int ensure_frontier_buffers(lbm_ctx *c)
{
    if (c->pmark) return LBM_OK;
    const size_t nb = (size_t)c->nblocks;
    struct {
        void **dst;
        size_t bytes;
    } want[] = {
        {(void **)&c->pmark, nb * sizeof(unsigned)},  {(void **)&c->plist, nb * sizeof(int)},
        {(void **)&c->pcount, sizeof(int)},           {(void **)&c->pnsnap, sizeof(int)},
        {(void **)&c->pfeat, nb * LBM_MLP_IN * sizeof(float)}, {(void **)&c->pprob, nb * sizeof(float)},
        {(void **)&c->prep, nb * sizeof(unsigned)},   {(void **)&c->nbits_pre, nb * CELLS * sizeof(uint32_t)},
    };
    for (auto &w : want) {
        *w.dst = dev_alloc(c, w.bytes);
        if (!*w.dst) return fail(c, LBM_ENOMEM, "device allocation of %zu bytes failed", w.bytes);
    }
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->prep, 0, nb * sizeof(unsigned), c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_frontier_features(lbm_ctx *c, int32_t *blocks, float *feat, long long cap, long long *n)
{
    if (!c || !n) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    if (cap > 0 && (!blocks || !feat)) return fail(c, LBM_EINVAL, "blocks and feat are required");
    if (c->kp.shape != 0) return fail(c, LBM_EINVAL, "frontier features are defined for 8x8x8 blocks");
    DeviceGuard g(c->device);
    int rc = ensure_frontier_buffers(c);
    if (rc) return rc;
    if (c->side) CUDA_OR_FAIL(c, cudaStreamSynchronize(c->side));
    KParams &k = c->kp;
    cudaStream_t s = c->stream;
    const int t = (int)c->step;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->pnsnap, &k.ctrl->n_active[t & 1], sizeof(int),
                                    cudaMemcpyDeviceToDevice, s));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->pmark, 0, c->nblocks * sizeof(unsigned), s));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->pcount, 0, sizeof(int), s));
    CUDA_OR_FAIL(c, launch_frontier(k, c->pnsnap, c->pmark, c->plist, c->pcount, c->sms, s));
    CUDA_OR_FAIL(c, launch_features(k, t & 1, c->pnsnap, c->plist, c->pcount, c->pfeat, c->sms, s));
    c->launches += 2;
    int cnt = 0;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(&cnt, c->pcount, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    *n = cnt;
    if (cap <= 0 || cnt == 0) return LBM_OK;
    std::vector<int> list(cnt);
    std::vector<float> f((size_t)cnt * LBM_MLP_IN);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(list.data(), c->plist, cnt * sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(f.data(), c->pfeat, f.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    std::vector<int> order(cnt);
    for (int i = 0; i < cnt; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return list[a] < list[b]; });
    const long long m = std::min<long long>(cap, cnt);
    for (long long i = 0; i < m; ++i) {
        blocks[i] = list[order[i]];
        std::memcpy(feat + i * LBM_MLP_IN, f.data() + (size_t)order[i] * LBM_MLP_IN, LBM_MLP_IN * sizeof(float));
    }
    return LBM_OK;
}

int lbm_activation_steps(lbm_ctx *c, int32_t *out)
{
    if (!c || !out) return LBM_EINVAL;
    if (!c->geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry has not been called");
    DeviceGuard g(c->device);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(out, c->kp.act_step, c->nblocks * sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_proposer(lbm_ctx *c, lbm_mlp *mlp, int period, float threshold)
{
    if (!c) return LBM_EINVAL;
    if (mlp && c->kp.shape != 0) return fail(c, LBM_EINVAL, "the activation proposer needs 8x8x8 blocks");
    DeviceGuard g(c->device);
    drop_graph(c);
    if (!mlp) {
        if (c->side) CUDA_OR_FAIL(c, cudaStreamSynchronize(c->side));
        c->mlp = nullptr;
        c->kp.prep = nullptr;
        c->kp.nbits_pre = nullptr;
        return LBM_OK;
    }
    if (!c->p.progressive) return fail(c, LBM_EINVAL, "the proposer needs the progressive mesh");
    if (period < 1) return fail(c, LBM_EINVAL, "period must be >= 1");
    if (!std::isfinite(threshold)) return fail(c, LBM_EINVAL, "threshold must be finite");
    int rc = ensure_frontier_buffers(c);
    if (rc) return rc;
    if (!c->side) {
        CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&c->side_ev, cudaEventDisableTiming));
        CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&c->side_done, cudaEventDisableTiming));
    }
    c->mlp = mlp;
    c->period = period;
    c->threshold = threshold;
    c->kp.prep = c->prep;
    c->kp.nbits_pre = c->nbits_pre;
    return LBM_OK;
}

int lbm_set_exec(lbm_ctx *c, int mode)
{
    if (!c) return LBM_EINVAL;
    if (mode != LBM_EXEC_STREAM && mode != LBM_EXEC_GRAPH && mode != LBM_EXEC_PERSISTENT &&
        mode != LBM_EXEC_STAGED)
        return fail(c, LBM_EINVAL, "unknown execution mode %d", mode);
    DeviceGuard g(c->device);
    if (c->kp.aa && (mode == LBM_EXEC_PERSISTENT || mode == LBM_EXEC_STAGED))
        return fail(c, LBM_EINVAL, "A-A streaming runs in the STREAM and GRAPH modes");
    if (mode == LBM_EXEC_PERSISTENT) {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
        if (!coop) return fail(c, LBM_EINVAL, "the device has no cooperative launch");
    }
    c->exec = mode;
    c->kp.staged = mode == LBM_EXEC_STAGED ? 1 : 0;
    drop_graph(c);
    return LBM_OK;
}

int lbm_set_slot_order(lbm_ctx *c, int period)
{
    if (!c) return LBM_EINVAL;
    if (period < 0) return fail(c, LBM_EINVAL, "period must be >= 0");
    c->sort_period = period;
    return LBM_OK;
}

int lbm_set_slot_strip(lbm_ctx *c, int rows)
{
    if (!c) return LBM_EINVAL;
    if (rows < -1) return fail(c, LBM_EINVAL, "rows must be >= -1");
    c->strip_rows = rows;
    c->kp.strip = rows < 0 ? auto_strip(c->nbx, c->nby) : (rows >= c->nby ? 0 : rows);
    drop_graph(c);
    return LBM_OK;
}

int lbm_set_fusion(lbm_ctx *c, int on, int max_lag)
{
    if (!c) return LBM_EINVAL;
    if (on != 0 && on != 1) return fail(c, LBM_EINVAL, "on must be 0 or 1");
    if (max_lag < 0) return fail(c, LBM_EINVAL, "max_lag must be >= 0");
    c->fuse = on != 0;
    c->kp.fz_max_lag = max_lag;
    drop_graph(c);
    return LBM_OK;
}

int lbm_set_density_partials(lbm_ctx *c, int on)
{
    if (!c) return LBM_EINVAL;
    if (on != 0 && on != 1) return fail(c, LBM_EINVAL, "on must be 0 or 1");
    c->partials = on != 0;
    // the next pass 1 pulls; the partials are written again by the next collision
    c->part_ok = false;
    drop_graph(c);
    return LBM_OK;
}

int lbm_barrier_selftest(int missing, long long spins)
{
    if (missing < 0 || spins < 1) return LBM_EINVAL;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return barrier_selftest(missing, spins, sms);
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err : g_create_error; }

}  // extern "C"
