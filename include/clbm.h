/*
 * clbm.h -- C ABI of the GB300 (sm_103a) D2Q9 cascaded lattice Boltzmann
 * library with the consistent forcing scheme of
 *   L. Fei and K. H. Luo, "Consistent forcing scheme in the cascaded lattice
 *   Boltzmann method", arXiv:1705.11092 (Phys. Rev. E 96, 053307, 2017).
 * Section, equation and remark numbers below refer to that paper.
 *
 * Conventions (all entry points):
 *   - Every call returns a clbm_status (0 = CLBM_OK, negative = error) and
 *     never aborts or prints.  clbm_status_string() names a status.
 *   - Host arrays are row-major with node index y * nx + x (x fastest);
 *     population arrays are 9 planes [9][ny][nx] in the velocity order of
 *     Eq. 1: e_x = {0,1,0,-1,0,1,-1,-1,1}, e_y = {0,0,1,0,-1,1,1,-1,-1}.
 *   - Inputs are copied; the caller keeps ownership of every pointer it
 *     passes.  Outputs are caller-allocated.
 *   - Work is queued on the context's CUDA stream (the caller's stream if
 *     one was given to clbm_create, else a private non-blocking stream).
 *     Calls that return host data synchronise that stream; clbm_step and the
 *     *_dev calls are asynchronous.
 *   - After a device-side or CUDA error the context holds a sticky error;
 *     later calls return CLBM_ERR_STATE until clbm_destroy.
 *   - A context is not thread-safe.
 *
 * The lattice is periodic in x and y.  Walls are solid nodes with halfway
 * bounce-back (Sec. 4A): a population that would stream from a fluid node
 * into a solid node returns to the fluid node with the opposite velocity at
 * the next step, so the wall lies half-way between the two nodes.
 *
 * The stored state of a context is the post-collision population field
 * f*(x, t) of Eq. 9/12 after the last step; one clbm_step pulls f* from the
 * neighbours (Eq. 10, pull form), which is the pre-collision f(x, t+1), and
 * collides it (Eq. 12).  Populations are stored as shifted deviations
 * g_i = (f_i - w_i rho0) * 2^k in the chosen format (rho0 = 1, w_i the D2Q9
 * weights, k the per-run scale exponent, 0 except for FP16).
 */
#ifndef CLBM_H
#define CLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct clbm_ctx clbm_ctx;

/* Storage format of the populations.  FP64 computes in FP64; FP32, FP16 and
 * BF16 compute in FP32 in deviation form. */
typedef enum { CLBM_FP64 = 0, CLBM_FP32 = 1, CLBM_FP16 = 2, CLBM_BF16 = 3 } clbm_format;

/* Shape of the body force F of Eq. 12-15. */
typedef enum {
    CLBM_FORCE_UNIFORM = 0, /* (fx, fy) everywhere; `force` ignored           */
    CLBM_FORCE_ROWS = 1,    /* force = [ny][2] (Fx, Fy) per row y             */
    CLBM_FORCE_COLUMNS = 2, /* force = [nx][2] (Fx, Fy) per column x          */
    CLBM_FORCE_FIELD = 3,   /* force = [ny][nx][2] per node                   */
    CLBM_FORCE_SHAN_CHEN = 4 /* force = [3] (G, psi0, rho0): the Shan-Chen
                              * interaction force of Sec. 4C, recomputed from
                              * the density field before every collision      */
} clbm_force_kind;

/* Forcing scheme of the collision.  CLBM_FORCING_CONSISTENT is the paper's
 * scheme (Eq. 12-15); M1 (Premnath et al., Eq. 17-20) and M2 (Lycett-Brown
 * and Luo, Eq. 21) are the schemes it is compared with in Sec. 3-4. */
typedef enum {
    CLBM_FORCING_CONSISTENT = 0,
    CLBM_FORCING_M1 = 1,
    CLBM_FORCING_M2 = 2
} clbm_forcing;

typedef enum {
    CLBM_OK = 0,
    CLBM_ERR_ARG = -1,      /* invalid argument                               */
    CLBM_ERR_OOM = -2,      /* device allocation failed                       */
    CLBM_ERR_CUDA = -3,     /* a CUDA call or kernel failed                   */
    CLBM_ERR_DIVERGED = -4, /* a reduction found NaN or Inf                   */
    CLBM_ERR_TIMEOUT = -5,  /* a device-side wait gave up                     */
    CLBM_ERR_STATE = -6     /* sticky error from an earlier call              */
} clbm_status;

/*
 * Create a lattice.  Sec. 2 (Eq. 1-15) defines the step it runs.
 *   out        receives the context (owned by the library; free with
 *              clbm_destroy).  Set to NULL on error.
 *   nx, ny     lattice size, each >= 2 (>= 3 in y and x if any node is solid).
 *   rates      diag(S) of Eq. 7 in the order (s0, s1, s1, sb, s2, s2, s3, s3,
 *              s4); each in (0, 2); entries 1-2, 4-5 and 6-7 must be equal.
 *              s0 and s1 do not affect the result (Remark 5).
 *   force_kind clbm_force_kind; `force` is the matching host FP64 array (or
 *              NULL for CLBM_FORCE_UNIFORM), (fx, fy) the uniform force.
 *              CLBM_FORCE_SHAN_CHEN (Sec. 4C): force = {G, psi0, rho0} with
 *              psi0 > 0; before every collision the force is
 *                F(x) = -G psi(x) sum_i w_i psi(x + e_i) e_i,
 *              psi = psi0 exp(-rho0 / rho) of the node densities (Eq. 11),
 *              w_i = 1/3 on the axes and 1/12 on the diagonals (G < 0
 *              attracts; the paper's liquid-vapour case is G = -10/3,
 *              psi0 = rho0 = 1).  The lattice must have no solid node; each
 *              step then also runs a density pass over the lattice (see
 *              clbm_bytes_per_update).  Batches do not take this kind.
 *   solid      host [ny][nx], nonzero = solid node; NULL = all fluid.
 *   format     clbm_format of the stored populations.
 *   stream     cudaStream_t to run on (e.g. torch's current stream), or NULL
 *              for a private stream.
 * The state is f* of the rest equilibrium rho = 1, u = 0 until clbm_init or
 * clbm_set_populations.  Errors: CLBM_ERR_ARG, CLBM_ERR_OOM, CLBM_ERR_CUDA.
 */
int clbm_create(clbm_ctx** out, int nx, int ny, const double rates[9], int force_kind,
                const double* force, double fx, double fy, const uint8_t* solid, int format,
                void* stream);

/*
 * Initialise with the generalized local equilibrium of (rho, u) (Sec. 2A,
 * Eq. 8: its central moments are [rho,0,0,2 rho cs^2,0,0,0,0,rho cs^4]) as the
 * pre-collision state at t = 0, then collide it once (Eq. 12).  rho, ux, uy
 * are host FP64 [ny][nx]; NULL rho means 1 everywhere, NULL ux/uy mean 0.
 * Values at solid nodes are ignored.  For FP16 the scale exponent is chosen
 * here from the largest deviation (see clbm_scale_exponent).  When every
 * given input is page-locked memory mapped into the device's address space
 * (as cudaHostAlloc'd memory is), the kernel reads it in place; otherwise
 * the fields pass through a device staging buffer.  Returns after the state
 * is in place.
 */
int clbm_init(clbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* As clbm_init with device FP64 arrays (e.g. torch tensors); asynchronous. */
int clbm_init_dev(clbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/*
 * Set the state from host FP64 f[9][ny][nx]; values at solid nodes are
 * ignored.
 *   pre_collision = 1: f is a pre-collision state f(x, t); it is collided
 *                      once (Eq. 12) and the result stored.
 *   pre_collision = 0: f is a post-collision state f*(x, t) (as
 *                      clbm_get_populations returns it); it is stored as
 *                      given, with no collision.  A state read with
 *                      pre_collision = 0 and set back this way continues
 *                      the run (checkpoint and resume): bit for bit for
 *                      FP16 and BF16 storage and for FP32 deviations of
 *                      magnitude above 2^-31, to FP64 round-off for FP64
 *                      storage.  FP16 encodes with the current scale
 *                      exponent (clbm_scale_exponent).
 * Errors: CLBM_ERR_ARG (NULL f, pre_collision not 0 or 1), CLBM_ERR_OOM.
 */
int clbm_set_populations(clbm_ctx* ctx, const double* f, int pre_collision);

/*
 * Read the state, decoded to FP64, into host f[9][ny][nx]; solid nodes
 * read as 0.
 *   pre_collision = 0: the stored post-collision state f*(x, t) (Eq. 9/12).
 *   pre_collision = 1: the pre-collision state f(x, t+1) that the next step
 *                      collides: f*(x, t) pulled from the neighbours
 *                      (Eq. 10), f_i(x) = f*_i(x - e_i), and where x - e_i
 *                      is solid the halfway bounce-back value f*_opp(i)(x)
 *                      (Sec. 4A).  The density and velocity of Eq. 11 and
 *                      Eq. 15 are defined on this state.
 * Errors: CLBM_ERR_ARG (NULL f, pre_collision not 0 or 1), CLBM_ERR_OOM.
 */
int clbm_get_populations(clbm_ctx* ctx, double* f, int pre_collision);

/*
 * Read a w-by-h window of the stored post-collision state, decoded to FP64,
 * into host f[9][h][w]: entry (i, j, k) is node ((x0 + k) mod nx,
 * (y0 + j) mod ny).  0 <= x0 < nx, 0 <= y0 < ny, w, h >= 1.  Solid nodes
 * read as 0.  Used for sampled checks of lattices too large to copy whole.
 */
int clbm_get_window(clbm_ctx* ctx, int x0, int y0, int w, int h, double* f);

/*
 * clbm_get_window, enqueued only: the readout kernel and the copy into host
 * f[9][h][w] follow the work already on the lattice's stream, and the call
 * returns without waiting.  The values are in f once the stream has passed
 * the copy (clbm_synchronize, or an event the caller records on that stream
 * after this call); f must stay valid until then.  Page-locked f that is
 * mapped into the device's address space (as cudaHostAlloc'd memory is) is
 * written directly by the readout kernel; other f goes through a device
 * staging buffer and a copy, which the CUDA runtime makes synchronous for
 * pageable memory.  With page-locked f a loop can read each step's result
 * while the next step runs.  Reads in flight share one device staging
 * buffer in stream order (it grows, after draining the stream, when a larger
 * window is asked for).  Errors: as clbm_get_window.
 */
int clbm_get_window_async(clbm_ctx* ctx, int x0, int y0, int w, int h, double* f);

/*
 * Advance n >= 0 time steps: pull-stream with halfway bounce-back (Eq. 10,
 * Sec. 4A), density and velocity (Eq. 11, 15), central moments (Eq. 4-6),
 * relaxation with consistent forcing (Eq. 7, 8, 12, 14), back-transform
 * (Eq. 9), all in one fused kernel launch per step.  Asynchronous.
 */
int clbm_step(clbm_ctx* ctx, int n);

/*
 * Density and velocity of the current time level (Eq. 11, Eq. 15) from the
 * stored post-collision state: rho = sum f*_i, rho u = sum f*_i e_i - F/2
 * (the collision adds F to the momentum, Eq. 12).  Host FP64 [ny][nx];
 * any pointer may be NULL; solid nodes give 0.  When every given output is
 * page-locked memory mapped into the device's address space (as
 * cudaHostAlloc'd memory is), the kernel writes it directly; otherwise the
 * fields pass through a device staging buffer and copies.  Returns after
 * the values are in place.
 */
int clbm_moments(clbm_ctx* ctx, double* rho, double* ux, double* uy);

/* As clbm_moments into device FP64 arrays; asynchronous. */
int clbm_moments_dev(clbm_ctx* ctx, double* rho, double* ux, double* uy);

/*
 * FP64 reductions over the fluid nodes, in a fixed order (deterministic):
 * out[0] = total mass sum rho, out[1], out[2] = total momentum sum rho u
 * (Eq. 11, 15).  Returns CLBM_ERR_DIVERGED if any sum is NaN or Inf.
 * `out` is host memory (3 doubles); synchronises the stream.
 */
int clbm_reduce(clbm_ctx* ctx, double out[3]);

/*
 * Relative L2 velocity error E_2 of Eq. 24 against a reference field, over
 * the fluid nodes, accumulated in FP64 on the device.  ua, va are host FP64
 * [ny][nx].  `out` receives E_2.
 */
int clbm_l2_error(clbm_ctx* ctx, const double* ua, const double* va, double* out);

/*
 * Select the forcing scheme (clbm_forcing; default CLBM_FORCING_CONSISTENT).
 * M1 (Eq. 17-19): T~* = (I-S)(T~) + S(T~eq - C_P/2), f* = M^-1 N^-1 T~* +
 * Delta f, with Delta f the distribution whose central moments are
 * C_P = [0,Fx,Fy,0,...,0]; this equals Eq. 12 without the third-order
 * forcing moments.  M2 (Eq. 21): the forcing moments are (1 - s2/2) N M R_G
 * with Guo's R_G (Remark 3); momentum is kept only when s1 = s2 (Remark 5).
 * Takes effect for the next collision (clbm_init, clbm_set_populations or
 * clbm_step).  Errors: CLBM_ERR_ARG.
 */
int clbm_set_forcing_scheme(clbm_ctx* ctx, int scheme);

/* Wait for all queued work of the context; reports asynchronous errors. */
int clbm_synchronize(clbm_ctx* ctx);

/*
 * Scale exponent k of the stored deviations (g = (f - w rho0) 2^k); 0 except
 * for FP16.  clbm_set_scale_exponent sets it before the next init (0..40).
 */
int clbm_scale_exponent(const clbm_ctx* ctx);
int clbm_set_scale_exponent(clbm_ctx* ctx, int k);

/*
 * Launch shape of the step kernel (no effect on the results' definition):
 *   vec_bytes  bytes each lane moves per population plane, 16 or 8 (FP64:
 *              16 only); smaller vectors halve the per-thread registers.
 *   packed     FP32-compute formats: 1 = collide two nodes per packed FP32x2
 *              instruction, 0 = one node per FP32 instruction.  Both round
 *              every operation identically (bit-identical results).
 *   prefetch   0..4: how many task strides ahead each warp asks L2 for its
 *              next rows (0 = no prefetch); direct-load kernel only.
 *   stages     0 = each warp loads its rows straight into registers; 2 or 3
 *              = each warp keeps a ring of that many row chunks in shared
 *              memory, filled by asynchronous copies issued ahead of use.
 * Defaults: FP64 (16, 0, 0, 0); FP32, FP16, BF16 (16, 1, 0, 2).  Takes
 * effect at the next clbm_step.  Any
 * out-of-range value gives CLBM_ERR_ARG and leaves the shape unchanged.
 */
int clbm_set_tuning(clbm_ctx* ctx, int vec_bytes, int packed, int prefetch, int stages);
int clbm_get_tuning(const clbm_ctx* ctx, int* vec_bytes, int* packed, int* prefetch, int* stages);

/*
 * Task form of lattices with solid nodes (no effect on others).  By default
 * a warp takes a chunk of 32 consecutive vectors of a row (vec_bytes each
 * per plane).  With CLBM_SPARSE_ON it instead takes 32 consecutive entries of
 * the list of vectors that hold at least one fluid node (row-major), so no
 * lane idles on an all-solid vector; the list's tasks whose vectors are all
 * plain (no fluid node beside a solid one, no solid node) run without the
 * bounce-back work, in a launch of their own; with a staged launch shape,
 * the rows with no solid node within one step, when they are at least an
 * eighth of the rows, leave the list and run the unmasked row-chunk step
 * over a list of rows.  CLBM_SPARSE_AUTO (default)
 * uses the list when fewer than 90 % of the vectors hold a fluid node, and
 * for FP16 and BF16 lattices of 2^23 nodes or more.  The list
 * costs 8 bytes per listed vector, its entry and the vector's bounce-back
 * plan (built on the host with the list), and one read of each per step
 * (of the plan, only by the tasks with bounce-back work); it is rebuilt by
 * clbm_set_tuning when the vector width changes.  Lattices wider than
 * 65536 vectors or taller than 65536 rows, and M2 lattices, keep the chunk
 * form.  Results do not depend on the form (bit for bit).  Errors:
 * CLBM_ERR_ARG (unknown mode), CLBM_ERR_OOM.
 */
typedef enum { CLBM_SPARSE_OFF = 0, CLBM_SPARSE_ON = 1, CLBM_SPARSE_AUTO = 2 } clbm_sparse;

/*
 * Rounding of the populations the time step stores (FP16 and BF16 only; the
 * paper fixes no storage precision).  CLBM_ROUND_NEAREST (default) rounds to
 * nearest even.  With CLBM_ROUND_STOCHASTIC a value between two
 * representable neighbours is rounded up with probability equal to its
 * distance from the lower one, so a change smaller than half a storage step
 * (a small body force's increment per step, for instance) is kept on
 * average instead of being dropped every step.  The random bits come from a
 * hash of the node, the population and a step counter kept on the device
 * (it starts at 0 when this mode is first set): a run is reproducible, and
 * every launch shape and CUDA-graph replay gives the same bits.  The
 * rounding itself is the GPU's stochastic-rounding conversion (16 random
 * bits per value).  One rounding errs by less than one storage step
 * instead of half a step.  The counter adds one single-thread launch per
 * step.  Initialisation
 * (clbm_init, clbm_set_populations) still rounds to nearest.  Errors:
 * CLBM_ERR_ARG (unknown mode; stochastic mode for FP64/FP32), CLBM_ERR_OOM.
 */
typedef enum { CLBM_ROUND_NEAREST = 0, CLBM_ROUND_STOCHASTIC = 1 } clbm_rounding;
int clbm_set_rounding(clbm_ctx* ctx, int mode);
int clbm_set_sparse(clbm_ctx* ctx, int mode);
/* Number of sparse tasks in use (0: chunk tasks). */
int clbm_sparse_tasks(const clbm_ctx* ctx);

/* Algorithmic HBM bytes one fluid-node update moves (18 populations, plus
 * 1 byte of bounce-back link bits and 1 bit of solid flag when the lattice
 * has solid nodes; Shan-Chen lattices: 27 populations and the psi value
 * written and read, in the compute type), and the fluid-node count. */
double clbm_bytes_per_update(const clbm_ctx* ctx);
long long clbm_fluid_nodes(const clbm_ctx* ctx);

/* Lattice size of a context (either pointer may be NULL).  Errors:
 * CLBM_ERR_ARG (NULL ctx). */
int clbm_get_size(const clbm_ctx* ctx, int* nx, int* ny);

/*
 * Test hook for the library's failure paths (no counterpart in the paper):
 * the next device allocation of the library in this process
 * (CLBM_FAIL_ALLOC), or the next time-step launch (CLBM_FAIL_LAUNCH), reports
 * failure as if CUDA had returned an out-of-memory or a launch error; the
 * failed call sends nothing to the GPU.  A failed allocation returns
 * CLBM_ERR_OOM and leaves the context or batch as it was, still usable (a
 * failed clbm_create or clbm_batch_create returns no handle).  A failed
 * launch returns CLBM_ERR_CUDA and makes the error sticky: later calls on
 * that context or batch return CLBM_ERR_STATE until it is destroyed.  The
 * hook fires once; CLBM_FAIL_NONE clears it.  Errors: CLBM_ERR_ARG.
 */
typedef enum { CLBM_FAIL_NONE = 0, CLBM_FAIL_ALLOC = 1, CLBM_FAIL_LAUNCH = 2 } clbm_fail;
int clbm_debug_fail_next(int what);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices (each its own size, rates, force and
 * walls, one storage format) advanced together.  Every time step is one
 * fused launch of the step kernel over all lattices (a flat list of row
 * chunks), so small lattices share the GPU with large ones; steps are
 * replayed from CUDA graphs.  Each lattice runs exactly the step of
 * clbm_step (Sec. 2, Eq. 1-15, halfway bounce-back of Sec. 4A): a lattice's
 * result in a batch equals its result run alone, bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct clbm_batch clbm_batch;

/* One lattice of a batch; the fields mean what clbm_create's arguments of
 * the same names mean.  Pointed-to arrays are copied at creation. */
typedef struct {
    int nx, ny;
    double rates[9];
    int force_kind;
    const double* force;
    double fx, fy;
    const uint8_t* solid;
    int forcing;            /* clbm_forcing of this lattice */
} clbm_domain_desc;

/*
 * Create a batch of `count` >= 1 lattices in one storage format, on
 * `stream` (NULL: private stream).  Each lattice starts at f* of the rest
 * equilibrium.  Errors: CLBM_ERR_ARG (any lattice fails clbm_create's
 * checks, a forcing value is not a clbm_forcing, or the batch would have
 * 2^31 or more row chunks of 64 nodes: sum of ny * ceil(nx / 64) over the
 * lattices), CLBM_ERR_OOM, CLBM_ERR_CUDA.
 */
int clbm_batch_create(clbm_batch** out, int count, const clbm_domain_desc* domains, int format,
                      void* stream);

/* Per-lattice counterparts of clbm_init, clbm_set_populations,
 * clbm_get_populations, clbm_moments, clbm_reduce and clbm_l2_error for
 * lattice `domain` (0 <= domain < count); same layouts and semantics. */
int clbm_batch_init(clbm_batch* b, int domain, const double* rho, const double* ux,
                    const double* uy);
int clbm_batch_set_populations(clbm_batch* b, int domain, const double* f, int pre_collision);
int clbm_batch_get_populations(clbm_batch* b, int domain, double* f, int pre_collision);
int clbm_batch_moments(clbm_batch* b, int domain, double* rho, double* ux, double* uy);
int clbm_batch_reduce(clbm_batch* b, int domain, double out[3]);
int clbm_batch_l2_error(clbm_batch* b, int domain, const double* ua, const double* va,
                        double* out);

/* Advance every lattice by n >= 0 steps (asynchronous; a persistent
 * launch's timeout surfaces at the next synchronising call). */
int clbm_batch_step(clbm_batch* b, int n);

/* How the warps of a batched step share the flat list of (lattice, row,
 * chunk) tasks: CONTIGUOUS gives each warp one range of the list (a warp
 * meets few lattices); INTERLEAVED gives warp w the tasks w, w + W, w + 2W,
 * ... for W warps (all warps sweep the batch together, as one band of
 * rows). */
typedef enum { CLBM_SCHEDULE_CONTIGUOUS = 0, CLBM_SCHEDULE_INTERLEAVED = 1 } clbm_schedule;

/*
 * Launch shape of the batched step: vec_bytes 16 or 8, packed 0 or 1,
 * stages 0, 2 or 3 (see clbm_set_tuning; FP64 accepts only vec_bytes 16,
 * packed 0), schedule a clbm_schedule.  Results do not depend on it
 * (bit for bit).  A task is 32 consecutive vectors of one lattice in
 * row-major order (it may run on into the next row), so ragged row ends
 * leave no lanes idle.
 * Defaults: FP64 (16, 0, 0, INTERLEAVED); FP32, FP16, BF16
 * (16, 1, 2, CONTIGUOUS).  Any other value returns CLBM_ERR_ARG.
 */
int clbm_batch_set_tuning(clbm_batch* b, int vec_bytes, int packed, int stages, int schedule);
int clbm_batch_get_tuning(const clbm_batch* b, int* vec_bytes, int* packed, int* stages,
                          int* schedule);

/*
 * How batched steps are launched (results do not depend on it, bit for
 * bit):
 *   persistent 0: one launch per time step, the launch boundary being the
 *                 step barrier (default).
 *              1: one cooperative launch advances many steps (up to 32 per
 *                 launch, replayed from CUDA graphs).  The warps split the
 *                 flat task list into contiguous ranges, and between steps
 *                 a warp waits only for the lattices it works on: each
 *                 lattice counts the warps that finished it at the current
 *                 step, and a warp starts the lattice's next step once all
 *                 of them have.  Every wait polls a bounded number of times
 *                 (clbm_batch_set_wait); one that gives up leaves a status
 *                 that the next synchronising call returns as
 *                 CLBM_ERR_TIMEOUT (then the batch is sticky).  Tasks that
 *                 lie inside a lattice's longest run of rows with no solid
 *                 node within one step run the step without the masks.
 *                 Needs a staged launch shape (stages 2 or 3) and no M2
 *                 lattice.
 *   resident   1 (persistent only): the smallest lattices whose state fits
 *                 twice in a block's shared-memory stage (at most 128, and
 *                 never every lattice) are each held in one block's shared
 *                 memory for a whole launch, read from and written to
 *                 device memory once per launch instead of once per step.
 *   order      0: the flat task list follows the lattices in the given
 *                 order; 1: largest lattices first.
 * Errors: CLBM_ERR_ARG (values, or persistent with stages 0 or an M2
 * lattice, or resident without persistent).
 */
int clbm_batch_set_mode(clbm_batch* b, int persistent, int resident, int order);
int clbm_batch_get_mode(const clbm_batch* b, int* persistent, int* resident, int* order);

/* Number of lattices held in shared memory by the current mode. */
int clbm_batch_resident_lattices(const clbm_batch* b);

/*
 * Bound of the waits of persistent launches: each gives up after
 * spin_limit polls (0 <= spin_limit < 2^32; default 2^20, about a second),
 * a poll being one acquire load of the lattice's counter and a short sleep.
 * delay_ns (0 .. 10^8) is a test hook: the first streaming warp of every
 * persistent launch starts that many nanoseconds late, so that together
 * with a small spin_limit a wait is sure to give up.  Takes effect at the
 * next step.  Errors: CLBM_ERR_ARG.
 */
int clbm_batch_set_wait(clbm_batch* b, long long spin_limit, long long delay_ns);

/*
 * Autotuner: times launch shapes for `steps` steps each on this batch (CUDA
 * events on the batch's stream): first every vector width x packing x ring
 * depth x schedule with one launch per step, then, around the fastest, the
 * largest-first lattice order and the persistent launches (ring depth x
 * lattices held in shared memory or not x order).  It keeps the fastest
 * and remembers it for batches of the same GPU, format and lattice shapes:
 * in this process, and across processes in a text file (CLBM_TUNE_CACHE if
 * set, an empty value for none; else $XDG_CACHE_HOME/clbm-batch-tuning.txt
 * or ~/.cache/clbm-batch-tuning.txt; a file that cannot be written is
 * skipped).  If ms_per_step is NULL and the shape is remembered, it is
 * applied without timing; otherwise *ms_per_step receives the best time.
 * Timing advances the batch, so tune before initialising.
 */
int clbm_batch_autotune(clbm_batch* b, int steps, double* ms_per_step);

int clbm_batch_synchronize(clbm_batch* b);

/* Fluid nodes of the whole batch; algorithmic HBM bytes of one batch step
 * (per lattice: fluid nodes times clbm_bytes_per_update's figure). */
long long clbm_batch_fluid_nodes(const clbm_batch* b);
double clbm_batch_bytes_per_step(const clbm_batch* b);
int clbm_batch_scale_exponent(const clbm_batch* b, int domain);

/* Destroy a batch (NULL-safe). */
int clbm_batch_destroy(clbm_batch* b);

/*
 * No counterpart in the paper: a library service for callers that cannot
 * allocate device memory (an embedding framework that owns every device
 * byte through its own pool or budget, a latency-critical loop where an
 * allocation and the synchronisation it may imply are not allowed, or code
 * that never creates a context because creating one allocates).
 *
 * FP64 totals of a post-collision population field the caller holds in
 * device memory, the same sums clbm_reduce returns: out[0] = sum rho,
 * out[1], out[2] = sum rho u (rho = sum f*_i, rho u = sum f*_i e_i - F/2,
 * Eq. 11, 15), out[3] = number of nodes with a non-finite value.  Fixed
 * summation order (deterministic).  This call allocates nothing: it calls
 * no cudaMalloc, cudaFree or allocating library routine.
 *   f       device FP64 [9][ny][nx] populations (the layout of
 *           clbm_get_populations), read only.
 *   nx, ny  lattice size; nx >= 1, 1 <= ny <= CLBM_NOALLOC_MAX_ROWS.
 *   fx, fy  uniform body force.
 *   solid   device uint8 [ny][nx], nonzero = solid node (skipped), or NULL.
 *   out     device, 4 doubles, written (not accumulated).
 *   stream  cudaStream_t to run on; NULL = the legacy default stream.
 * Asynchronous on `stream`.  Its scratch is a fixed 2 MiB device array
 * (CLBM_NOALLOC_MAX_ROWS slots of 4 doubles) in the library's device code;
 * the driver commits it on a device when it loads that code there, which
 * under lazy module loading (CUDA's default) is this call's first use on
 * the device, and keeps it until the context is destroyed.  ny beyond the
 * maximum gives CLBM_ERR_ARG.  The first call on a device, and the first
 * after its context was recreated, looks up the array's device address
 * there (make that call before any stream capture).
 * All calls share the array and it keeps the last call's values; each call
 * overwrites every slot it reads, so nothing needs clearing, but calls that
 * overlap on the GPU (different streams, or devices sharing the slots via
 * peer access) race: order them.
 * Errors: CLBM_ERR_ARG (NULL f or out, bad sizes, non-finite force),
 * CLBM_ERR_CUDA.
 */
#define CLBM_NOALLOC_MAX_ROWS 65536
int clbm_reduce_noalloc(const double* f, int nx, int ny, double fx, double fy,
                        const uint8_t* solid, double* out, void* stream);

/*
 * Measured arithmetic throughput of the current device (no counterpart in
 * the paper; the arithmetic roofs of the step kernels): kind 0 = FP64 fused
 * multiply-add, 1 = FP32 fused multiply-add, 2 = packed FP32x2 fused
 * multiply-add (two per instruction), 3 = FP64 add, 4 = FP64 multiply.
 * Every SM runs 2048 threads of 8 independent chains, for at least
 * `seconds` (0 < seconds <= 60) by CUDA events; *ops_per_second receives
 * operations per second (one per lane and value; an FMA is two flops).
 * Allocates a small output buffer and a stream for the measurement.
 * Errors: CLBM_ERR_ARG, CLBM_ERR_OOM, CLBM_ERR_CUDA.
 */
int clbm_alu_throughput(int kind, double seconds, double* ops_per_second);

/* Destroy a context (NULL-safe); frees its device memory. */
int clbm_destroy(clbm_ctx* ctx);

/* Static string naming a status code. */
const char* clbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CLBM_H */
