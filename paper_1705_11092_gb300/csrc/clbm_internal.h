// clbm_internal.h -- host-side interface between the C ABI (clbm_api.cu) and
// the kernels (clbm_kernels.cu, clbm_reduce.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace clbm {

template <class C> struct Relax;

// Collision constants (Eq. 7, 12, 14 and the forcing scheme) in both
// compute precisions: om_b, om_2, om_3, om_4, sb23, s4_9, f3, g1, c2, m2
// (see Coef in clbm_device.cuh).
struct RelaxBoth {
    double d[10];
    float f[10];
};

// Geometry of one lattice in device memory.
struct Geometry {
    int nx, ny;
    int pitch;          // elements per stored row (multiple of the vector width)
    long long plane;    // elements per population plane = ny * pitch
};

// Arguments of the fused step kernel.
// Fields of a sparse list's info word (vector_info in clbm_host.h): solid
// flags in bits 0-7, then the all-solid source rows, the own vectors held in
// plane slots, the other own vectors, whether links 1 and 3 bounce, which
// neighbour elements the warp-edge lanes fetch, and the not-plain flag.
constexpr uint32_t kInfoRowShift = 8, kInfoCoverShift = 11, kInfoRestShift = 17,
                   kInfoBounce1 = 23, kInfoBounce3 = 24, kInfoLeftShift = 25,
                   kInfoRightShift = 28, kInfoNotPlain = 1u << 31;
static_assert(kInfoRightShift == kInfoLeftShift + 3, "edge bits follow the edge slots");

struct StepArgs {
    const void* src;         // post-collision planes at t   [9][ny][pitch]
    void* dst;               // post-collision planes at t+1 [9][ny][pitch]
    const uint8_t* lmask;    // link bits [ny][pitch] or null (no solid nodes)
    const uint8_t* sbits;    // solid bitmap, bit (y*pitch + x) of byte >> 3; null iff lmask is
    Geometry geo;
    int vec_bytes;           // bytes per lane and plane: 16 or 8 (FP64: always 16)
    int packed;              // FP32 compute: 1 = two nodes per packed FP32x2 op
    int prefetch;            // L2 prefetch distance in task strides (0 = none)
    int stages;              // 0 = direct loads; 2, 3 = shared-memory cp.async ring depth
    int chunks;              // 32-lane row chunks per row (batched steps: vectors per
                             // row, tasks of 32 consecutive vectors)
    int sround;              // 16-bit storage: 1 = stochastic rounding of the step's stores
    long long ntasks;        // ny * chunks (batched: ceil(ny * chunks / 32))
    const uint32_t* vlist;   // sparse single-lattice steps: the vectors with a fluid
                             // node (row << 16 | vector), padded with 0xffffffff to
                             // 32 vtasks entries; null = regular (row, chunk) tasks
    const uint32_t* vinfo;   // sparse lists: one word per entry of vlist, the
                             // vector's solid flags and bounce-back plan (see
                             // vector_info in clbm_host.h)
    const int* rowlist;      // sparse lists: rows whose vectors are all plain (no solid
                             // node within one step), stepped by the unmasked row-chunk
                             // kernel; their vectors are not in vlist
    int vtasks;
    int nrows;               // entries of rowlist
    int plain_y0, plain_y1;  // batched steps: rows [plain_y0, plain_y1) hold only plain
                             // vectors (no link bit, no solid node); tasks inside
                             // them run the unmasked step
    int ptasks;              // sparse lists: the first ptasks tasks hold plain vectors
                             // (no link bit, no solid node), stepped without the
                             // bounce-back and solid-node work
    int force_kind;          // clbm_force_kind
    const void* force;       // force array in the compute type, or null
    double fx, fy;           // uniform force
    const void* psi;         // Shan-Chen: psi field [ny][pitch] in the compute type
    double sc_g;             // Shan-Chen interaction strength G
    double sc_psi0, sc_rho0; // Shan-Chen pseudopotential psi = psi0 exp(-rho0 / rho)
    const uint32_t* sr_step; // device step counter seeding the rounding hash
    double rho0;             // reference density of the deviation shift
    double scale, inv_scale; // 2^k and 2^-k
    RelaxBoth relax;
    // derived on the host from fx, fy, scale and sc_g (derive_args), so that
    // an FP32-compute step does no FP64 arithmetic per chunk: the run scale,
    // the scaled uniform force and G in each compute type
    double fxs_d, fys_d;
    float scale_f, fxs_f, fys_f, sc_g_f;
};

// Link bits: bit i-1 (i = 1..8) of lmask[y*pitch + x] is set when the node
// x - e_i is solid (exact for every node, solid or fluid).  The solid flag of
// node (x, y) is bit (q & 7) of sbits[q >> 3], q = y*pitch + x.  Padding
// columns are solid with every link bit set.

// format: 0 FP64, 1 FP32, 2 FP16, 3 BF16 (clbm_format)
int element_size(int format);
// nodes per lane for a format and vector size
int vector_width_of(int format, int vec_bytes);

cudaError_t launch_step(const StepArgs& a, int format, cudaStream_t s);
// one per format (clbm_step_<format>.cu)
cudaError_t launch_step_fp64(const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32(const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp16(const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_bf16(const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp16sr(const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_bf16sr(const StepArgs& a, cudaStream_t s);
// advance the stochastic-rounding step counter (one thread)
cudaError_t launch_sr_tick(uint32_t* counter, cudaStream_t s);

// Equilibrium of (rho, ux, uy) (device FP64 [ny][nx], null = defaults) as the
// pre-collision state, collided once, encoded into dst.
cudaError_t launch_init(const StepArgs& a, int format, const double* rho, const double* ux,
                        const double* uy, cudaStream_t s);
// FP64 state f [9][ny][nx] (device) into a.dst: collide = 1, a pre-collision
// state collided once; collide = 0, a post-collision state stored as given.
cudaError_t launch_set_populations(const StepArgs& a, int format, const double* f, int collide,
                                   cudaStream_t s);
// Decoded state (FP64 [9][ny][nx], device) of a.src: pre = 0 the stored
// post-collision state, pre = 1 the pre-collision state pulled from it.
cudaError_t launch_get_populations(const StepArgs& a, int format, double* f, int pre, cudaStream_t s);
// Decoded post-collision populations of a periodic window (FP64 [9][h][w]).
cudaError_t launch_window(const StepArgs& a, int format, int x0, int y0, int w, int h,
                          double* out, cudaStream_t s);
// rho, ux, uy (device FP64 [ny][nx], any may be null) of a.src.
cudaError_t launch_moments(const StepArgs& a, int format, double* rho, double* ux, double* uy,
                           cudaStream_t s);
// Shan-Chen pseudopotential field psi[ny][pitch] (compute type, device) of
// a lattice without solid nodes.  mode 0: from the density of the
// pre-collision state the next step pulls out of a.src; mode 1: from the
// density of the stored state a.src itself (the one its last collision used).
cudaError_t launch_psi(const StepArgs& a, int format, int mode, void* psi, cudaStream_t s);
// The same field for an initial state given on the device: kind 0 from the
// density field rho (null: 1), kind 1 from FP64 populations f [9][ny][nx].
cudaError_t launch_psi_prepare(const StepArgs& a, int format, int kind, const double* rho,
                               const double* f, void* psi, cudaStream_t s);
// Largest |deviation| of a.src, as a double into *out (device), for the scale choice.
cudaError_t launch_max_abs_dev(const StepArgs& a, int format, double* out, cudaStream_t s);

// One lattice of a batch: its description (src = copy A, dst = copy B of
// its populations) for the batched step kernel.
struct BatchDomain {
    StepArgs a;
};

// Arguments of one batched step launch.
struct BatchLaunch {
    const BatchDomain* doms;   // device, ndom entries
    const int* task0;          // device, first flat task of each lattice
    int ndom;
    int ntasks;                // < 2^31 (checked when the batch is created)
    int parity;                // 0: A -> B, 1: B -> A
    int vec_bytes, packed;
    int stages;                // 0 = direct loads; 2, 3 = shared-memory ring depth
    int guo;                   // some lattice uses the M2 forcing scheme
    int schedule;              // 0: contiguous task range per warp; 1: interleaved
    int mask_mode;             // lattices with solid nodes: 0 none, 1 all, 2 some
    // persistent launches (persist = 1): one cooperative launch advances
    // nsteps steps (parity is that of the first); a warp waits only for the
    // lattices it works on, through per-lattice counters, with bounded polls
    int persist;
    int nsteps;
    int nres;                  // lattices doms[ndom .. ndom + nres - 1] are held in
                               // shared memory for the launch ...
    int res_blocks;            // ... by blocks 0 .. res_blocks - 1: block r takes
    const int* res_first;      // lattices ndom + res_first[r] .. ndom + res_first[r + 1] - 1
    unsigned* done;            // device [ndom]: warps that finished the lattice's current
                               // step (zeroed by the launch)
    int* status;               // device: 0, or 1 once a wait gave up
    unsigned spin_limit;       // polls before a wait gives up
    unsigned delay_ns;         // test hook: the first streaming warp starts this much later
};

// Dynamic shared memory of a block of the staged batch kernels (the ring of
// its warps), the space a lattice held in shared memory must fit twice.
size_t batch_stage_bytes(int format, int vec_bytes, int stages, int mask_mode);

cudaError_t launch_batch_step(const BatchLaunch& b, int format, cudaStream_t s);

// Device allocation of the library, with the test hook of
// clbm_debug_fail_next (clbm_api.cu).
cudaError_t dev_alloc(void** p, size_t bytes);
template <class T> cudaError_t dev_alloc(T** p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void**>(p), bytes);
}
// True (once) when the hook asks the next step launch to fail.
bool take_launch_failure();
cudaError_t launch_batch_step_fp64(const BatchLaunch& b, cudaStream_t s);
cudaError_t launch_batch_step_fp32(const BatchLaunch& b, cudaStream_t s);
cudaError_t launch_batch_step_fp16(const BatchLaunch& b, cudaStream_t s);
cudaError_t launch_batch_step_bf16(const BatchLaunch& b, cudaStream_t s);

// FP64 reductions (clbm_reduce.cu).  partials: device scratch of
// reduce_partials_count() * 4 doubles; out: device, 4 doubles.
int reduce_partials_count();
// sums over fluid nodes of (rho, rho ux, rho uy, nonfinite flag)
cudaError_t launch_reduce_moments(const StepArgs& a, int format, double* partials, double* out,
                                  cudaStream_t s);
// sums of ((u-ua)^2 + (v-va)^2, ua^2 + va^2) over fluid nodes
cudaError_t launch_reduce_l2(const StepArgs& a, int format, const double* ua, const double* va,
                             double* partials, double* out, cudaStream_t s);

}  // namespace clbm
