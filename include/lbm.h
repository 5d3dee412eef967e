/*
 * liblbm: progressive-mesh, two-component pseudo-potential lattice
 * Boltzmann time step (D3Q19) on one GB300 GPU (sm_103a).
 *
 * Method: Duchateau et al., "A Progressive Mesh Method for Physical
 * Simulations Using Lattice Boltzmann Method on Single-Node multi-GPU
 * Architectures" (arXiv:1510.03560).
 *   - SRT-BGK lattice Boltzmann equation and equilibrium: Sec. 2.1, Eqs. 1-5.
 *   - Peng-Robinson EOS, pseudo-potential, cohesion, inter-component and
 *     extra (gravity, fluid-solid) forces, exact-difference forcing:
 *     Sec. 2.2, Eqs. 6-12.
 *   - Progressive mesh: sub-domains created where the velocity-change
 *     criterion of Eq. 13 exceeds S on the boundary of the meshed region:
 *     Sec. 4.1-4.3, Fig. 4.
 *   - Throughput metric (MLUPS): Sec. 5.3, Eq. 16.
 *
 * The sub-domain (the unit of meshing) is a block of 512 cells, 8 x 8 x 8
 * by default (lbm_params.block selects 16 x 8 x 4, 16 x 4 x 8 or
 * 32 x 4 x 4).  A block is "active" once meshed; blocks are never removed.
 * Unmeshed blocks behave as a resting ambient at the densities rho_amb.
 *
 * Conventions shared by every entry point:
 *   - Grid arrays are dense, x fastest: index x + nx * (y + ny * z).
 *   - Per-component arrays are [ncomp][nz][ny][nx]; velocity arrays
 *     [ncomp][3][nz][ny][nx].
 *   - Cell types: 0 fluid, 1 solid (halfway bounce-back wall), 2 held (its
 *     populations stay at the initial equilibrium: inlets, outlets).
 *   - Block ids are linear, x fastest: bx + nbx * (by + nby * bz), with
 *     nbx = nx / (block extent along x) and so on.
 *   - Host pointers belong to the caller and are only read or written
 *     during the call; the library never keeps them.
 *   - The context owns all device memory it allocates (through the
 *     caller's allocator when one is given) and frees it in lbm_destroy.
 *   - Every function returns LBM_OK or an error code; the message of the
 *     last error is available from lbm_last_error().  No exception or
 *     process exit crosses this interface.  A context is used by one host
 *     thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_EINVAL 1  /* invalid argument or parameter */
#define LBM_ENOMEM 2  /* block pool full, or a device allocation failed */
#define LBM_ECUDA 3   /* a CUDA runtime call failed */
#define LBM_ESTATE 4  /* call out of order (e.g. lbm_step before lbm_set_geometry) */
#define LBM_ETIMEOUT 5 /* a bounded device wait gave up (grid barrier of LBM_EXEC_PERSISTENT) */

/* How lbm_step enqueues the steps (lbm_set_exec); every mode runs the same
 * per-cell code and gives the same results bit for bit. */
#define LBM_EXEC_STREAM 0     /* one launch per step for pass 1, one for the collision
                                 (or one for both, fused: lbm_set_fusion), plus block
                                 creation's two (default) */
#define LBM_EXEC_GRAPH 1      /* the launches of two steps captured once as a CUDA graph,
                                 replayed (the kernels read the step count on the device) */
#define LBM_EXEC_PERSISTENT 2 /* the steps of a call in one cooperative launch, with grid
                                 barriers between the phases (waits bounded: LBM_ETIMEOUT) */
#define LBM_EXEC_STAGED 3     /* as STREAM, with each block's populations brought into shared
                                 memory by one bulk (TMA) copy, double buffered (FP32 with
                                 two components; other forms run as STREAM) */

#define LBM_CELL_FLUID 0
#define LBM_CELL_SOLID 1
#define LBM_CELL_HELD 2

/* Storage form of the populations (lbm_params.storage).  Arithmetic is FP32
 * in every form.  The 16-bit forms store each population as its deviation
 * f_i - w_i rho_r from the resting equilibrium of rho_r, the density that
 * the cell which will read the value (the cell x + e_i, or x itself behind a
 * solid wall) had at the step the value was written; a reader adds w_i
 * times its own previous density back; the rest population is written
 * from the decoded values of the others, so a cell's mass is unchanged by
 * their rounding.  This is not part of the paper; it halves the population
 * traffic of Eqs. 1 and 10.  Measured against the FP64 method: FP16 within
 * 1e-3 relative density; BF16 within 1e-3 except next to a strongly driven
 * density jump (up to 2e-3 in the first fluid layers behind a held liquid
 * inlet into gas). */
#define LBM_STORAGE_FP32 0
#define LBM_STORAGE_FP16 1 /* IEEE binary16 deviations */
#define LBM_STORAGE_BF16 2 /* bfloat16 deviations */

/* Streaming pattern of the populations (lbm_params.streaming; Sec. 3
 * compares the A-B pattern, two arrays read and written alternately, with
 * the A-A pattern, one array updated in place, which the paper uses to
 * halve the memory of the populations).  Both give the same results bit for
 * bit.  A-A needs the FP32 storage form with two components and the STREAM
 * or GRAPH execution mode. */
#define LBM_STREAM_AB 0
#define LBM_STREAM_AA 1

#define LBM_BLOCK_EDGE 8 /* cells per block edge of the default 8^3 block */
#define LBM_Q 19         /* D3Q19 populations per component */

typedef struct lbm_ctx lbm_ctx;

/* Device allocator: returns a device pointer of at least `bytes` bytes
 * (256-byte aligned) or NULL; `user` is lbm_params.alloc_user. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *user);
typedef void (*lbm_free_fn)(void *ptr, void *user);

typedef struct lbm_params {
    int nx, ny, nz;      /* grid, each a positive multiple of the block extent */
    int ncomp;           /* 1 or 2; component 0 follows the Peng-Robinson EOS,
                            component 1 is an ideal gas (p = rho / 3, psi = 0) */
    int periodic[3];     /* per axis: 1 wraps around, 0 ends in solid cells */
    int progressive;     /* 1: progressive mesh (Sec. 4); 0: static mesh, every
                            block holding a non-solid cell meshed from the start */
    int storage;         /* LBM_STORAGE_FP32 (0), _FP16 or _BF16 */
    int streaming;       /* LBM_STREAM_AB (0) or LBM_STREAM_AA */
    int block[3];        /* cells per block along x, y, z (the paper's sub-domain
                            shape, Sec. 4.1): 8x8x8 (default; {0, 0, 0} selects it),
                            16x8x4, 16x4x8 or 32x4x4.  Shapes other than 8^3 need the
                            FP32 storage form and no activation proposer. */
    double tau;          /* BGK relaxation time, Eq. 1 (> 0.5) */
    double beta;         /* weighting term of Eq. 8 (the paper uses 1.16) */
    double pr_a, pr_b, pr_R, pr_omega; /* Peng-Robinson a, b, R, acentric factor, Eq. 7 */
    double T_over_Tc;    /* temperature as a fraction of Tc = 0.0778 a / (0.45724 b R) */
    double g_self;       /* g_aa of Eqs. 6 and 8 (< 0 attracts; 0 turns cohesion off) */
    double g_cross;      /* g_aa' of Eq. 9 (> 0 repels) */
    double g_ads[2];     /* fluid-solid strength per component: F = -g_ads *
                            max(0, rho - rho_amb) * sum_i w_i s(x + e_i) e_i */
    double grav[3];      /* body-force acceleration: F = (rho - rho_ref) * grav */
    double rho_ref[2];   /* reference density of the body force, per component */
    double S;            /* threshold of Eq. 13 (>= 0): a block is created when
                            ||u(t) - u(t-1)||_2 > S at a neighbouring cell */
    long long max_blocks; /* block-pool capacity in blocks; 0 = every block */
    lbm_alloc_fn dev_alloc; /* NULL: cudaMallocAsync on `stream` */
    lbm_free_fn dev_free;
    void *alloc_user;
    void *stream;        /* cudaStream_t for every launch and copy; NULL = default */
} lbm_params;

/* Counters of a context (lbm_get_stats). */
typedef struct lbm_stats {
    long long steps;            /* completed time steps */
    long long active_blocks;    /* blocks meshed now */
    long long capacity;         /* block-pool capacity */
    long long total_blocks;     /* blocks of the grid */
    long long nonsolid_blocks;  /* blocks holding at least one non-solid cell */
    long long cell_updates;     /* sum over completed steps of 512 x active blocks */
    long long fluid_updates;    /* sum over completed steps of the fluid cells of active blocks */
    long long launches;         /* kernels this context has launched */
    long long device_bytes;     /* device memory held by the context */
    double kernel_ms[4];        /* with profiling on: device time per kernel kind
                                   (0 stream+macro, 1 block creation, 2 force+collide,
                                   3 other) accumulated over lbm_step calls */
    long long kernel_launches[4];
    long long created_blocks;   /* blocks created by the criterion since lbm_set_geometry */
    long long prepared_blocks;  /* blocks the activation proposer prepared */
    long long prepared_hits;    /* created blocks that had been prepared */
    long long slot_sorts;       /* renumberings of the meshed slots in block order */
    long long fused_deferred;   /* fused step: pass-1 work items deferred to the end of
                                   their launch (their neighbourhood's collisions came
                                   later in the work order), summed over launches */
    long long fused_waited;     /* fused step: pass-1 items that found a neighbouring
                                   collision still running and waited for it */
    long long fused_lag_distance; /* fused step: the slot distance its lag covers now */
} lbm_stats;

/* Validate `p`, allocate the block pool (capacity x 2 buffers x ncomp x 19 x
 * 512 populations of 4 bytes, or 2 in the 16-bit storage forms; one buffer
 * with A-A streaming) and the tables, and return a new context in *out.
 * The pool holds the sub-domains of Sec. 4.1 (here 8^3-cell blocks, or the
 * other block shapes): the domain is not meshed all at once, blocks are
 * taken from the pool as the fluid reaches them (Sec. 4.2-4.3), and
 * max_blocks bounds how many can exist (Fig. 3).
 * Allocates through p->dev_alloc when given.  Errors: LBM_EINVAL (bad
 * parameter: grid not a multiple of 8, ncomp not 1 or 2, tau <= 0.5, S < 0,
 * unknown storage form or streaming pattern, A-A streaming without the FP32
 * form and two components, ...; no CUDA call is made then), LBM_ENOMEM,
 * LBM_ECUDA.  On error *out is NULL. */
int lbm_create(const lbm_params *p, lbm_ctx **out);

/* Free everything the context holds (the sub-domain pool of Sec. 4.1 and
 * its tables).  Waits for the context's stream first.  NULL is accepted. */
int lbm_destroy(lbm_ctx *ctx);

/* Geometry and initial state (Sec. 4.1: the first sub-domains are created
 * where the fluid starts).
 *   cell_type  [nz][ny][nx] uint8, values 0..2 (see above)
 *   rho_init   [ncomp][nz][ny][nx] initial densities
 *   u_init     [ncomp][3][nz][ny][nx] initial velocities, or NULL for rest
 *   rho_amb    [ncomp] densities of the resting ambient in unmeshed blocks
 * The initial populations are the equilibrium of Eq. 2 at (rho_init,
 * u_init).  Progressive mode meshes every block that holds a non-solid cell
 * whose initial state differs from the ambient; static mode meshes every
 * block holding a non-solid cell.  Held cells must sit in meshed blocks or
 * hold exactly the ambient state.  Resets the step counter.  Errors:
 * LBM_EINVAL, LBM_ENOMEM (initial blocks exceed the capacity), LBM_ECUDA. */
int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *cell_type, const float *rho_init,
                     const float *u_init, const float *rho_amb);

/* Advance `nsteps` time steps and wait for them.  One step: pull
 * streaming and the macroscopic moments (Eqs. 4-5) on the meshed blocks;
 * in progressive mode the criterion of Eq. 13 on cells bordering unmeshed
 * blocks and the creation of the blocks it selects (they start from the
 * ambient equilibrium and take part in the same step); Peng-Robinson psi
 * (Eqs. 6-7); forces (Eqs. 8-9, gravity, fluid-solid); forced BGK collision
 * (Eqs. 10-12).  Errors: LBM_ESTATE (no geometry, or an earlier error),
 * LBM_ENOMEM (the pool cannot hold the blocks a step creates: the state is
 * left as it was after the last completed step, and stepping stays refused),
 * LBM_ECUDA. */
int lbm_step(lbm_ctx *ctx, int nsteps);

/* lbm_step without the final wait: enqueues the steps on the context's
 * stream and returns.  Errors raised on the device (LBM_ENOMEM) are
 * reported by the next lbm_sync. */
int lbm_step_async(lbm_ctx *ctx, int nsteps);

/* Wait for enqueued work and report its status (as lbm_step). */
int lbm_sync(lbm_ctx *ctx);

/* Macroscopic fields of component `comp` for the current state: the
 * density of Eq. 4 and, for fluid cells, the velocity u + F / (2 rho) (the
 * velocity of the exact-difference forcing scheme), both as the next step
 * would compute them after streaming.  Held cells report the moments of
 * their own populations, solid cells 0, cells of unmeshed blocks the
 * ambient density at rest.  Outputs: host arrays of nx*ny*nz floats (any
 * of the four may be NULL).  Errors: LBM_EINVAL, LBM_ESTATE, LBM_ECUDA. */
int lbm_get_macro(lbm_ctx *ctx, int comp, float *rho, float *ux, float *uy, float *uz);

/* Ids of the meshed blocks in ascending order: the sub-domains created so
 * far (Sec. 4.1, Fig. 3: the first ones at lbm_set_geometry, then those the
 * criterion of Eq. 13 added, Sec. 4.3).  Block id = bx + nbx (by + nby bz).
 * Writes min(n, cap) ids to `ids` (host, may be NULL when cap is 0) and the
 * count to *n (cap <= 0 writes no ids).  Errors: LBM_EINVAL (ctx or n NULL,
 * or ids NULL with cap > 0), LBM_ESTATE (no geometry), LBM_ECUDA. */
int lbm_active_blocks(lbm_ctx *ctx, int32_t *ids, long long cap, long long *n);

/* Per-component mass: the density of Eq. 4 (the sum of a cell's
 * populations) summed over every non-solid cell, unmeshed cells counted at
 * the ambient equilibrium.  Streaming, bounce-back and the collision's
 * rest population (taken from the mass balance) conserve it, so it is the
 * check of a run: accumulated in FP64 on the device, per block and then
 * over blocks in slot order, so the same state gives the same bits.  mass:
 * host array of ncomp doubles.  Errors: LBM_EINVAL, LBM_ESTATE (no
 * geometry), LBM_ECUDA. */
int lbm_mass(lbm_ctx *ctx, double *mass);

/* Post-collision populations of one meshed block, host array
 * [ncomp][19][512] in the library's velocity order (lbm_velocities), cell
 * index x + bx * (y + by * z) within a bx x by x bz block; in the 16-bit
 * storage forms the stored deviations with their reference added back, in
 * FP32, and 0 at solid cells (A-A streaming: 0 at solid cells as well).
 * LBM_EINVAL if the block is not meshed. */
int lbm_get_block_populations(lbm_ctx *ctx, int32_t block_id, float *out);

/* The library's D3Q19 velocity order: e[3 * i + axis], 19 x 3 ints. */
int lbm_velocities(int32_t *e);

/* Turn per-kernel device timing on (1) or off (0); on adds a pair of CUDA
 * events around each launch of lbm_step / lbm_step_async. */
int lbm_set_profiling(lbm_ctx *ctx, int on);

/* Counters; waits for enqueued work first. */
int lbm_get_stats(lbm_ctx *ctx, lbm_stats *out);

/* Message of the last error of `ctx`, or of the last failed lbm_create or
 * lbm_mass_noalloc (on the calling thread) when ctx is NULL.  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

#define LBM_NOALLOC_MAX_BLOCKS 65536 /* largest nblocks lbm_mass_noalloc accepts */

/* FP64 per-component mass of a population pool that the caller holds in
 * device memory, computed without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as a host application whose device memory is entirely
 * owned by another allocator (a framework that has reserved the whole GPU),
 * or a real-time loop that must not allocate after start-up.  Its scratch
 * (LBM_NOALLOC_MAX_BLOCKS x 2 partial sums and 2 totals, 1 MiB) is a
 * fixed-size array inside the library; every GPU that loads the library
 * holds it until the process exits.
 *   f        device pointer, [nblocks][ncomp][19][512] FP32 populations in the
 *            library's layout (velocity order of lbm_velocities, cell index
 *            x + 8 * (y + 8 * z) within a block); read only
 *   solid    device pointer, [nblocks][16] uint32 solid-cell bits (bit c % 32
 *            of word c / 32 set: cell c is solid and is left out), or NULL
 *   nblocks  1 .. LBM_NOALLOC_MAX_BLOCKS; larger is LBM_EINVAL
 *   ncomp    1 or 2
 *   mass     host array of ncomp doubles, written on success
 *   stream   cudaStream_t to run on (NULL = default stream); the call waits
 *            for it before returning
 * Each block's partial sum is formed as in lbm_mass (per cell over the 19
 * populations in order, then over the block's cells), and the partials are
 * added in row order.  So the result equals lbm_mass bit for bit when the
 * rows are every block of the grid in block order (none unmeshed, none fully
 * solid); otherwise it agrees to rounding.  Unlike lbm_mass it adds nothing
 * for blocks that are not passed (lbm_mass counts unmeshed blocks at the
 * ambient state).  Every call shares the one scratch array of its device and
 * rewrites every value it reads, so no state carries from one call to the
 * next; calls that overlap on the same GPU (other streams or host threads)
 * race on it and must be serialised by the caller.  Each call looks up the
 * array's device address on the current device (cudaGetSymbolAddress), so
 * the address stays valid after a cudaDeviceReset.  Errors: LBM_EINVAL,
 * LBM_ECUDA (message in lbm_last_error(NULL)). */
int lbm_mass_noalloc(const float *f, const uint32_t *solid, long long nblocks, int ncomp,
                     double *mass, void *stream);


/* Select LBM_EXEC_STREAM, _GRAPH or _PERSISTENT for later steps.  With
 * the proposer on, launches are split at its rounds.  With profiling on,
 * the device time of a graph or cooperative launch is counted as kind 3.
 * Errors: LBM_EINVAL (unknown mode, or no cooperative launch on the
 * device). */
int lbm_set_exec(lbm_ctx *ctx, int mode);

/* Slot order (progressive mesh).  A created block takes the next free slot
 * of the pool, so the slot order drifts from the spatial order and the
 * step's memory accesses lose locality.  Every `period` steps (default 64;
 * 0 = never) the device checks whether the blocks created since the last
 * renumbering reach 1/16 of the meshed ones and, if so, renumbers the meshed
 * slots in block order between two steps (moving the populations through
 * the idle population buffer; with A-A streaming, which has none, the
 * passes visit the slots in block order instead).  Results are the same bit
 * for bit with any period.  Errors: LBM_EINVAL (period < 0). */
int lbm_set_slot_order(lbm_ctx *ctx, int period);

/* Slot order of the block pool: the meshed slots are numbered in strips of
 * `rows` block rows along y, each strip in z, then y, then x order (0 = plain
 * block order, bx fastest; -1 = automatic, the default: strips of about 512
 * blocks per z layer, or block order when the grid is narrower).  A strip
 * keeps a block's z neighbours about rows * nbx slots away instead of
 * nbx * nby, so that the fused step's two passes meet within L2.  Applies at
 * the next lbm_set_geometry and at every renumbering.  Results are the same
 * bit for bit in every order.  Errors: LBM_EINVAL (rows < -1). */
int lbm_set_slot_strip(lbm_ctx *ctx, int rows);

/* Fused step (FP32 storage, two components, A-B streaming, STREAM and GRAPH
 * modes; off by default: on one GB300 it moves about 20 % fewer HBM bytes per
 * step but runs slower, pass 1 running at the collision's register budget).  The paper's step (Sec. 2, Eqs. 4-12) needs psi of
 * the 18 neighbours from the current step (Eqs. 6-9), so it is computed in
 * two passes over the meshed blocks: pass 1 streams the populations (Eq. 10,
 * left-hand side) for the densities, psi and the criterion (Eq. 13), pass 2
 * streams them again for the forces and the collision.  Fused, one launch
 * runs the collision of step t and, a lag behind it in the same work order,
 * pass 1 of step t + 1, which then reads the populations just written from
 * L2 rather than from HBM.  Pass 1 of a block waits (bounded; LBM_ETIMEOUT)
 * until the collisions of its 26 neighbours are written, or is deferred to
 * the end of the launch when one of them comes later in the work order.  The
 * results are the same bit for bit as unfused.  Between calls the next
 * step's pass 1 may already have run: lbm_get_macro, lbm_mass and the other
 * queries are unaffected.
 *   on       1 fused, 0 two launches per step
 *   max_lag  largest lag in half-block work items (0 = the default, 1536);
 *            below the neighbours' slot distance, more items are deferred
 * Errors: LBM_EINVAL (on not 0 or 1, max_lag < 0). */
int lbm_set_fusion(lbm_ctx *ctx, int on, int max_lag);

/* Density partials (FP32 storage, two components, A-B streaming; every
 * execution mode but LBM_EXEC_STAGED; off by default, unused while the fused
 * step is on: on one GB300 pass 1 moves 6.5x fewer HBM bytes and takes 40 %
 * less time, but the collision's shared-memory sums and barriers make it 50 %
 * slower, and the step about 20 % slower).  Pull streaming (Eq. 10, left-hand side) makes a cell's
 * density at step t + 1 the sum of the post-collision values of step t
 * that stream into it (Eq. 4), so the collision already holds every term.
 * Each half block of the collision sums, in shared memory, the terms its
 * cells pull from the half block itself (one value pair per cell) and the
 * terms it sends to each cell just outside its faces and edges (stored with
 * the receiving half block).  Pass 1 of step t + 1 then adds those few
 * values per cell for the densities and psi (Eqs. 4, 6, 7) instead of
 * pulling 38 populations; warps next to an unmeshed block still pull, since
 * the criterion (Eq. 13) needs their velocity.  The sums run in a fixed
 * order, so every mode and block order gives the same bits; against the
 * pull they differ only by the rounding of a reordered sum of 19 terms.
 * Meshed sets and fields still follow the FP64 oracle within the FP32
 * tolerances.  The first pass 1 after lbm_set_geometry, after switching
 * them on, or after a collision that did not write them pulls.
 *   on  1 partials, 0 pull in every pass 1
 * Errors: LBM_EINVAL (on not 0 or 1). */
int lbm_set_density_partials(lbm_ctx *ctx, int on);

/* Test hook of the bounded device wait: one cooperative launch whose grid
 * barrier expects `missing` more CTAs than it has, polling at most `spins`
 * times; returns the resulting status (LBM_OK when missing is 0,
 * LBM_ETIMEOUT otherwise) without affecting any context. */
int lbm_barrier_selftest(int missing, long long spins);

/* ---- learned activation proposer ------------------------------------------
 * Not part of the paper.  A small network predicts which unmeshed blocks the
 * criterion of Eq. 13 will create within the next steps; on a side stream
 * the context then prepares those blocks' per-cell solid words ahead of
 * time, work block creation would otherwise do when the block is created.
 * The criterion alone decides which blocks are created, and a prepared word
 * equals the one computed at creation, so results are bit-identical with
 * and without the proposer; a block that was not predicted is prepared at
 * creation as before.
 *
 * Features of a frontier block (an unmeshed block that is not all solid and
 * has a meshed face or edge neighbour), LBM_MLP_IN = 34 values:
 *   [0..1]   mean density of components 0 and 1 over the cells of its
 *            meshed face neighbours that touch it (rho_amb when none)
 *   [2..7]   mass flux into it through faces -x, +x, -y, +y, -z, +z: the
 *            sum over the touching cells of the neighbour of (j_0 + j_1) . n,
 *            n the unit normal into the block, j the momentum of Eq. 5 (0
 *            for an unmeshed neighbour)
 *   [8..33]  1 when the neighbour block (dx, dy, dz), dx fastest, skipping
 *            the block itself, is meshed, else 0
 * Moments are those of the next streaming of the current populations. */
#define LBM_MLP_IN 34
#define LBM_MLP_HIDDEN 64
/* parameters, packed: W1 [34][64], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 */
#define LBM_MLP_NPARAM (LBM_MLP_IN * LBM_MLP_HIDDEN + LBM_MLP_HIDDEN + \
                        LBM_MLP_HIDDEN * LBM_MLP_HIDDEN + LBM_MLP_HIDDEN + LBM_MLP_HIDDEN + 1)

/* Frontier blocks of the current state, ascending, and their features:
 * blocks [cap] int32, feat [cap][LBM_MLP_IN] (host arrays; either may be
 * NULL when cap is 0); *n receives the count (which may exceed cap). */
int lbm_frontier_features(lbm_ctx *ctx, int32_t *blocks, float *feat, long long cap,
                          long long *n);

/* Step at which each block was meshed: 0 for the initial blocks, t + 1 for
 * a block created by the criterion in step t (0-based), -1 for blocks not
 * meshed.  out: host array of nx/8 * ny/8 * nz/8 int32. */
int lbm_activation_steps(lbm_ctx *ctx, int32_t *out);

/* A multilayer perceptron LBM_MLP_IN -> 64 -> 64 -> 1 (ReLU, ReLU,
 * logistic output) with its own device memory, trained with the binary
 * cross-entropy.  Inputs are standardised inside: x' = (x - mean) * scale. */
typedef struct lbm_mlp lbm_mlp;

/* max_batch: the largest n of the calls below; stream: cudaStream_t (NULL =
 * default) for every launch.  Parameters start at zero, mean 0, scale 1. */
int lbm_mlp_create(int max_batch, void *stream, lbm_mlp **out);
int lbm_mlp_destroy(lbm_mlp *mlp);
/* params: host array of LBM_MLP_NPARAM floats, packed as above */
int lbm_mlp_set_params(lbm_mlp *mlp, const float *params);
int lbm_mlp_get_params(lbm_mlp *mlp, float *params);
/* mean, scale: host arrays of LBM_MLP_IN floats */
int lbm_mlp_set_scaling(lbm_mlp *mlp, const float *mean, const float *scale);
/* Probabilities prob[n] (device) of the n raw feature rows x [n][34]
 * (device).  bf16 = 1: inputs, hidden activations and weights rounded to
 * bfloat16, products accumulated in FP32; 0: FP32 throughout. */
int lbm_mlp_forward(lbm_mlp *mlp, const float *x, int n, int bf16, float *prob);
/* FP32 forward and backward pass over n rows x [n][34], labels y [n] (0 or
 * 1) (device): the mean loss to *loss (host) and its gradient with respect
 * to the parameters, kept for lbm_mlp_adam and copied to grad (host,
 * LBM_MLP_NPARAM floats) when grad is not NULL.  Every sum runs in a fixed
 * order, so the result does not depend on scheduling. */
int lbm_mlp_loss_grad(lbm_mlp *mlp, const float *x, const float *y, int n, double *loss,
                      float *grad);
/* One Adam update (step count t >= 1) with the last gradient. */
int lbm_mlp_adam(lbm_mlp *mlp, float lr, float beta1, float beta2, float eps, int t);

/* Use `mlp` (not owned; NULL turns the proposer off) every `period` steps
 * of lbm_step / lbm_step_async: frontier blocks whose probability (BF16
 * inference) exceeds `threshold` are prepared on a side stream.  The mlp
 * must outlive its use by the context.  Progressive mode and 8x8x8 blocks
 * only (LBM_EINVAL otherwise). */
int lbm_set_proposer(lbm_ctx *ctx, lbm_mlp *mlp, int period, float threshold);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
