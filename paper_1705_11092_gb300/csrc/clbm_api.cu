// clbm_api.cu -- the C ABI of include/clbm.h: lattice contexts, argument
// checks, device memory, the ping-pong buffers, CUDA-graph replay of the
// step loop, and host <-> device transfers around the kernels.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_device.cuh"
#include "clbm_host.h"
#include "clbm_internal.h"

using clbm::Geometry;
using clbm::RelaxBoth;
using clbm::StepArgs;

// steps captured per CUDA graph (even, so a replay keeps the buffer parity)
static const int kGraphSteps = 32;

struct clbm_ctx {
    int nx = 0, ny = 0, format = 0;
    Geometry geo{};
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;                        // buffer holding the current state
    uint8_t* lmask = nullptr;           // device link bits or null
    uint8_t* sbits = nullptr;           // device solid bitmap or null
    std::vector<uint8_t> solid_host;    // solid flags [ny][nx] (lattices with solid nodes)
    int sparse_mode = CLBM_SPARSE_AUTO; // clbm_set_sparse
    uint32_t* vlist = nullptr;          // device list of vectors holding a fluid node,
                                        // then (from vlist + vlist_cap) their info words
    size_t vlist_cap = 0;               // entries allocated
    int vtasks = 0;                     // > 0: sparse tasks in use
    int ptasks = 0;                     // of which the first hold plain vectors
    int* rowlist = nullptr;             // device list of the rows of plain vectors that
    int nrows = 0;                      // the row-chunk kernel steps (sparse lattices)
    int rowlist_cap = 0;
    int rounding = CLBM_ROUND_NEAREST;  // clbm_set_rounding
    uint32_t* sr_step = nullptr;        // device step counter of stochastic rounding
    int force_kind = 0;
    void* force = nullptr;              // device force array (compute type)
    double fx = 0.0, fy = 0.0;
    void* psi = nullptr;                // Shan-Chen psi field [ny][pitch] (compute type)
    double sc[3] = {0.0, 0.0, 0.0};     // Shan-Chen G, psi0, rho0
    double rates[9] = {0};
    RelaxBoth relax{};
    double rho0 = 1.0;
    int scale_k = 0;
    bool user_scale = false;
    int vec_bytes = 16;                 // launch shape of the step kernel (clbm_set_tuning)
    int packed = 0;
    int prefetch = 0;
    int stages = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap = nullptr;         // private stream for graph capture
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double* staging = nullptr;          // device FP64 staging for host transfers
    size_t staging_cap = 0;
    double* partials = nullptr;         // reduction scratch
    double* red_out = nullptr;
    long long fluid = 0;
    int sticky = CLBM_OK;
};

namespace clbm {

// Test hook of clbm_debug_fail_next: the failure the next device allocation
// or step launch of this process reports.
static std::atomic<int> g_fail_next{CLBM_FAIL_NONE};

cudaError_t dev_alloc(void** p, size_t bytes) {
    int want = CLBM_FAIL_ALLOC;
    if (g_fail_next.load() == CLBM_FAIL_ALLOC &&
        g_fail_next.compare_exchange_strong(want, CLBM_FAIL_NONE)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

bool take_launch_failure() {
    int want = CLBM_FAIL_LAUNCH;
    return g_fail_next.load() == CLBM_FAIL_LAUNCH &&
           g_fail_next.compare_exchange_strong(want, CLBM_FAIL_NONE);
}

}  // namespace clbm

namespace {

int fail(clbm_ctx* c, int status) {
    if (c && status == CLBM_ERR_CUDA) c->sticky = status;
    return status;
}

int cuda_status(clbm_ctx* c, cudaError_t e) {
    if (e == cudaSuccess) return CLBM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return CLBM_ERR_OOM;
    }
    return fail(c, CLBM_ERR_CUDA);
}

#define CLBM_CK(c, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_status(c, e_); \
    } while (0)

StepArgs make_args(const clbm_ctx* c, int src) {
    StepArgs a{};
    a.src = c->buf[src];
    a.dst = c->buf[src ^ 1];
    a.lmask = c->lmask;
    a.sbits = c->sbits;
    a.geo = c->geo;
    a.vec_bytes = c->vec_bytes;
    a.packed = c->packed;
    a.prefetch = c->prefetch;
    a.stages = c->stages;
    const int V = clbm::vector_width_of(c->format, c->vec_bytes);
    a.chunks = (c->nx + 32 * V - 1) / (32 * V);
    a.ntasks = (long long)c->ny * a.chunks;
    a.force_kind = c->force_kind;
    a.force = c->force;
    a.fx = c->fx;
    a.fy = c->fy;
    a.sround = c->rounding == CLBM_ROUND_STOCHASTIC;
    a.sr_step = c->sr_step;
    a.vlist = c->vtasks > 0 ? c->vlist : nullptr;
    a.rowlist = c->nrows > 0 ? c->rowlist : nullptr;
    a.nrows = c->nrows;
    a.vinfo = c->vtasks > 0 ? c->vlist + c->vlist_cap : nullptr;
    a.vtasks = c->vtasks;
    a.ptasks = c->ptasks;
    a.psi = c->psi;
    a.sc_g = c->sc[0];
    a.sc_psi0 = c->sc[1];
    a.sc_rho0 = c->sc[2];
    a.rho0 = c->rho0;
    a.scale = std::ldexp(1.0, c->scale_k);
    a.inv_scale = std::ldexp(1.0, -c->scale_k);
    a.relax = c->relax;
    clbm::derive_args(a);
    return a;
}

// The staging buffer of readouts; enqueued reads (clbm_get_window_async) may
// still be copying out of the old one, so the stream drains before it goes.
int ensure_staging(clbm_ctx* c, size_t doubles) {
    if (c->staging_cap >= doubles) return CLBM_OK;
    if (c->staging) {
        CLBM_CK(c, cudaStreamSynchronize(c->stream));
        cudaFree(c->staging);
    }
    c->staging = nullptr;
    c->staging_cap = 0;
    CLBM_CK(c, clbm::dev_alloc(&c->staging, doubles * sizeof(double)));
    c->staging_cap = doubles;
    return CLBM_OK;
}

bool shan_chen(const clbm_ctx* c) { return c->force_kind == CLBM_FORCE_SHAN_CHEN; }

// The sparse task list of a lattice with solid nodes (see clbm_set_sparse):
// every vector of V nodes that holds a fluid node, as row << 16 | vector,
// row-major, padded with 0xffffffff to whole tasks of 32 entries, the tasks
// of plain vectors first.  AUTO uses it when fewer than 90 % of the vectors
// hold a fluid node, where idle lanes cost time (measured on a 25 %-solid
// obstacle array against (row, chunk) tasks: FP64 +33 %, FP32 +3 %, FP16
// +7 %, FP16 with stochastic rounding +17 %), and for large 16-bit lattices.
int build_vlist(clbm_ctx* c) {
    c->vtasks = 0;
    c->ptasks = 0;
    c->nrows = 0;
    if (!c->lmask || c->sparse_mode == CLBM_SPARSE_OFF) return CLBM_OK;
    const int V = clbm::vector_width_of(c->format, c->vec_bytes);
    const int nvec = (c->nx + V - 1) / V;
    if (nvec > 65536 || c->ny > 65536) return CLBM_OK;        // entries hold 16-bit fields
    const int nx = c->nx, ny = c->ny;
    // rows with no solid node within one step (rows y - 1, y, y + 1): all
    // their vectors are plain.  With a shared-memory ring, when they are at
    // least an eighth of the rows, the unmasked row-chunk kernel steps them
    // over a list of rows and the vector list holds the other rows only
    // (8192 x 8193 channel: FP16 0.832 -> 0.869 of HBM, BF16 0.844 -> 0.882,
    // FP16 with stochastic rounding 0.786 -> 0.837; the obstacle array's
    // free rows run at the rate of the list's plain tasks either way).
    const std::vector<uint8_t> row_plain = clbm::plain_rows(c->solid_host.data(), nx, ny);
    std::vector<int> prows;
    for (int y = 0; y < ny; ++y)
        if (row_plain[y]) prows.push_back(y);
    const bool use_rows = c->stages > 0 && prows.size() * 8 >= (size_t)ny;
    // near[x] of row y: a solid node within one step of (x, y), periodic
    // (rows y - 1, y, y + 1 combined, then widened by one column)
    std::vector<uint8_t> rows3(nx), near(nx), links(nx);
    std::vector<uint32_t> all, info;
    std::vector<uint8_t> is_plain;
    long long nfluid_vec = 0;        // vectors holding a fluid node, rows of the row list included
    for (int y = 0; y < ny; ++y) {
        if (use_rows && row_plain[y]) {
            nfluid_vec += nvec;
            continue;
        }
        const uint8_t* r0 = c->solid_host.data() + (size_t)((y + ny - 1) % ny) * nx;
        const uint8_t* r1 = c->solid_host.data() + (size_t)y * nx;
        const uint8_t* r2 = c->solid_host.data() + (size_t)((y + 1) % ny) * nx;
        for (int x = 0; x < nx; ++x) rows3[x] = r0[x] | r1[x] | r2[x];
        for (int x = 0; x < nx; ++x)
            near[x] = rows3[x] | rows3[x == 0 ? nx - 1 : x - 1] | rows3[x == nx - 1 ? 0 : x + 1];
        bool have_links = false;     // the row's link bytes, built at its first non-plain vector
        for (int v = 0; v < nvec; ++v) {
            // the vectors holding a fluid node, row-major; plain ones have
            // their V nodes inside the row, fluid, with no solid neighbour
            bool fluid = false, p = v * V + V <= nx;
            for (int x = v * V; x < v * V + V && x < nx; ++x) {
                fluid |= r1[x] == 0;
                p = p && near[x] == 0;
            }
            if (!fluid) continue;
            ++nfluid_vec;
            all.push_back(((uint32_t)y << 16) | (uint32_t)v);
            if (!p && !have_links) {
                clbm::row_links(c->solid_host.data(), nx, ny, y, links.data());
                have_links = true;
            }
            info.push_back(p ? 0u : clbm::vector_info_row(links.data(), r1, nx, v, V));
            is_plain.push_back(p);
        }
    }
    // AUTO: the list where many vectors are all solid, and for 16-bit
    // storage on lattices far larger than L2 (there its plain tasks step
    // without the masked path's work: 8192^2 channel FP16 0.74 -> 0.83 of
    // HBM, with stochastic rounding 0.66 -> 0.79; FP32, which waits on
    // memory, is faster with row chunks, 0.94 against 0.90, and so are
    // small lattices, where the second launch per step shows)
    const double frac = (double)nfluid_vec / ((double)nvec * ny);
    const bool wide16 = (c->format == CLBM_FP16 || c->format == CLBM_BF16) && (long long)nx * ny >= (1LL << 23);
    if (c->sparse_mode == CLBM_SPARSE_AUTO && frac >= 0.9 && !wide16) return CLBM_OK;
    if (all.empty() && !use_rows) return CLBM_OK;
    if (use_rows) {
        if ((int)prows.size() > c->rowlist_cap) {
            if (c->rowlist) cudaFree(c->rowlist);
            c->rowlist = nullptr;
            c->rowlist_cap = 0;
            CLBM_CK(c, clbm::dev_alloc(&c->rowlist, prows.size() * sizeof(int)));
            c->rowlist_cap = (int)prows.size();
        }
        CLBM_CK(c, cudaMemcpyAsync(c->rowlist, prows.data(), prows.size() * sizeof(int), cudaMemcpyHostToDevice,
                                   c->stream));
        CLBM_CK(c, cudaStreamSynchronize(c->stream));
        c->nrows = (int)prows.size();
        if (all.empty()) return CLBM_OK;
    }
    all.resize((all.size() + 31) / 32 * 32, 0xffffffffu);
    info.resize(all.size(), 0u);
    is_plain.resize(all.size(), 0);
    // tasks of 32 consecutive entries; those whose vectors are all plain go
    // first (a task keeps its entries together, so a run of fluid nodes
    // between solids is read by one launch)
    std::vector<uint32_t> list, rest, linfo, rinfo;
    for (size_t t = 0; t < all.size(); t += 32) {
        bool p = true;
        for (size_t k = t; k < t + 32; ++k) p = p && is_plain[k];
        (p ? list : rest).insert((p ? list : rest).end(), all.begin() + t, all.begin() + t + 32);
        (p ? linfo : rinfo).insert((p ? linfo : rinfo).end(), info.begin() + t, info.begin() + t + 32);
    }
    c->ptasks = (int)(list.size() / 32);
    list.insert(list.end(), rest.begin(), rest.end());
    linfo.insert(linfo.end(), rinfo.begin(), rinfo.end());
    const size_t n = list.size();
    if (n > c->vlist_cap) {      // the entries, then as many info words
        if (c->vlist) cudaFree(c->vlist);
        c->vlist = nullptr;
        c->vlist_cap = 0;
        CLBM_CK(c, clbm::dev_alloc(&c->vlist, 2 * n * sizeof(uint32_t)));
        c->vlist_cap = n;
    }
    CLBM_CK(c, cudaMemcpyAsync(c->vlist, list.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                               c->stream));
    CLBM_CK(c, cudaMemcpyAsync(c->vlist + c->vlist_cap, linfo.data(), n * sizeof(uint32_t),
                               cudaMemcpyHostToDevice, c->stream));
    CLBM_CK(c, cudaStreamSynchronize(c->stream));
    c->vtasks = (int)(n / 32);
    return CLBM_OK;
}

// One time step from buffer src: for Shan-Chen lattices the psi field of the
// density the step will pull first, then the fused step.
cudaError_t launch_one_step(const clbm_ctx* c, int src, cudaStream_t s) {
    if (clbm::take_launch_failure()) return cudaErrorLaunchFailure;   // test hook: nothing launched
    if (shan_chen(c)) {
        cudaError_t e = clbm::launch_psi(make_args(c, src), c->format, 0, c->psi, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = clbm::launch_step(make_args(c, src), c->format, s);
    if (e == cudaSuccess && c->rounding == CLBM_ROUND_STOCHASTIC) e = clbm::launch_sr_tick(c->sr_step, s);
    return e;
}

// Before a readout that needs the force of the stored state (Eq. 15).
int psi_of_current(clbm_ctx* c) {
    if (shan_chen(c))
        CLBM_CK(c, clbm::launch_psi(make_args(c, c->cur), c->format, 1, c->psi, c->stream));
    return CLBM_OK;
}

void drop_graphs(clbm_ctx* c) {
    for (auto& g : c->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

int build_graph(clbm_ctx* c, int parity) {
    cudaGraph_t g = nullptr;
    CLBM_CK(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int src = parity;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < kGraphSteps && err == cudaSuccess; ++k) {
        err = launch_one_step(c, src, c->cap);
        src ^= 1;
    }
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(c, err);
    }
    CLBM_CK(c, e2);
    cudaError_t e3 = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    CLBM_CK(c, e3);
    return CLBM_OK;
}

int choose_scale(clbm_ctx* c) {
    // FP16 only: the run scale 2^k from the largest deviation
    if (c->format != CLBM_FP16 || c->user_scale) return CLBM_OK;
    c->scale_k = 0;
    double* dmax = c->red_out;
    CLBM_CK(c, cudaMemsetAsync(dmax, 0, sizeof(double), c->stream));
    StepArgs a = make_args(c, c->cur);
    CLBM_CK(c, clbm::launch_max_abs_dev(a, c->format, dmax, c->stream));
    double mx = 0.0;
    CLBM_CK(c, cudaMemcpyAsync(&mx, dmax, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CLBM_CK(c, cudaStreamSynchronize(c->stream));
    c->scale_k = clbm::fp16_scale_exponent(mx);
    return CLBM_OK;
}

int check_ctx(clbm_ctx* c) {
    if (!c) return CLBM_ERR_ARG;
    if (c->sticky != CLBM_OK) return CLBM_ERR_STATE;
    return CLBM_OK;
}

// The device address of page-locked host memory mapped into the device's
// address space (as cudaHostAlloc'd memory is), else null.
double* mapped_host(double* p) {
    if (!p) return nullptr;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
        return static_cast<double*>(pa.devicePointer);
    cudaGetLastError();                       // an unregistered pointer is not an error
    return nullptr;
}

}  // namespace

extern "C" {

const char* clbm_status_string(int status) {
    switch (status) {
        case CLBM_OK: return "ok";
        case CLBM_ERR_ARG: return "invalid argument";
        case CLBM_ERR_OOM: return "device allocation failed";
        case CLBM_ERR_CUDA: return "CUDA error";
        case CLBM_ERR_DIVERGED: return "non-finite value (diverged)";
        case CLBM_ERR_TIMEOUT: return "device wait timed out";
        case CLBM_ERR_STATE: return "context holds an earlier error";
    }
    return "unknown status";
}

int clbm_destroy(clbm_ctx* c) {
    if (!c) return CLBM_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (auto& b : c->buf)
        if (b) cudaFree(b);
    if (c->lmask) cudaFree(c->lmask);
    if (c->sbits) cudaFree(c->sbits);
    if (c->force) cudaFree(c->force);
    if (c->psi) cudaFree(c->psi);
    if (c->vlist) cudaFree(c->vlist);
    if (c->rowlist) cudaFree(c->rowlist);
    if (c->sr_step) cudaFree(c->sr_step);
    if (c->staging) cudaFree(c->staging);
    if (c->partials) cudaFree(c->partials);
    if (c->red_out) cudaFree(c->red_out);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return CLBM_OK;
}

int clbm_create(clbm_ctx** out, int nx, int ny, const double rates[9], int force_kind,
                const double* force, double fx, double fy, const uint8_t* solid, int format,
                void* stream) {
    if (!out) return CLBM_ERR_ARG;
    *out = nullptr;
    const int chk = clbm::check_lattice_args(nx, ny, rates, force_kind, force, fx, fy, format);
    if (chk != CLBM_OK) return chk;
    const bool sc = force_kind == CLBM_FORCE_SHAN_CHEN;
    if (sc && solid) {      // the Shan-Chen lattice has no solid nodes
        for (long long p = 0; p < (long long)nx * ny; ++p)
            if (solid[p]) return CLBM_ERR_ARG;
    }
    const size_t nforce = sc ? 0 : clbm::force_values(force_kind, nx, ny);

    clbm_ctx* c = new (std::nothrow) clbm_ctx();
    if (!c) return CLBM_ERR_OOM;
    c->nx = nx;
    c->ny = ny;
    c->format = format;
    std::memcpy(c->rates, rates, sizeof(c->rates));
    clbm::relax_constants(c->rates, CLBM_FORCING_CONSISTENT, c->relax);
    c->force_kind = force_kind;
    c->fx = fx;
    c->fy = fy;
    if (sc) std::memcpy(c->sc, force, sizeof(c->sc));
    // default launch shape, measured fastest on 8192^2 lattices: FP32-compute
    // formats collide node pairs in packed FP32x2 and stream through a 2-stage
    // shared-memory ring; FP64 (bound by FP64 arithmetic) loads directly.
    if (format != CLBM_FP64) {
        c->packed = 1;
        c->stages = 2;
    }
    const int esz = clbm::element_size(format);
    c->geo.nx = nx;
    c->geo.ny = ny;
    c->geo.pitch = clbm::row_pitch(nx, format);
    c->geo.plane = (long long)c->geo.pitch * ny;

    int st = CLBM_OK;
    auto bail = [&](int s) { clbm_destroy(c); return s == CLBM_ERR_CUDA ? CLBM_ERR_CUDA : s; };
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(CLBM_ERR_CUDA);
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(CLBM_ERR_CUDA);

    const size_t bytes = (size_t)9 * c->geo.plane * esz;
    for (auto& b : c->buf) {
        cudaError_t e = clbm::dev_alloc(&b, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); return bail(CLBM_ERR_OOM); }
        if (cudaMemsetAsync(b, 0, bytes, c->stream) != cudaSuccess) return bail(CLBM_ERR_CUDA);
    }
    if (clbm::dev_alloc(&c->partials, (size_t)clbm::reduce_partials_count() * 4 * sizeof(double)) != cudaSuccess ||
        clbm::dev_alloc(&c->red_out, 4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(CLBM_ERR_OOM);
    }
    if (sc) {
        const size_t csz = format == CLBM_FP64 ? sizeof(double) : sizeof(float);
        if (clbm::dev_alloc(&c->psi, (size_t)c->geo.pitch * ny * csz) != cudaSuccess) {
            cudaGetLastError();
            return bail(CLBM_ERR_OOM);
        }
    }

    // link bits and the solid bitmap (only when there are solid nodes)
    long long nsolid = 0;
    std::vector<uint8_t> m, sb;
    if (solid) nsolid = clbm::build_solid_masks(solid, nx, ny, c->geo.pitch, m, sb);
    c->fluid = (long long)nx * ny - nsolid;
    if (nsolid > 0) {
        if (clbm::dev_alloc(&c->lmask, m.size()) != cudaSuccess || clbm::dev_alloc(&c->sbits, sb.size()) != cudaSuccess) {
            cudaGetLastError();
            return bail(CLBM_ERR_OOM);
        }
        if (cudaMemcpy(c->lmask, m.data(), m.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->sbits, sb.data(), sb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(CLBM_ERR_CUDA);
        c->solid_host.resize((size_t)nx * ny);
        for (size_t p = 0; p < c->solid_host.size(); ++p) c->solid_host[p] = solid[p] != 0;
        if ((st = build_vlist(c))) return bail(st);
    }

    if (nforce) {
        std::vector<unsigned char> fb;
        clbm::force_in_compute_type(force, nforce, format, fb);
        if (clbm::dev_alloc(&c->force, fb.size()) != cudaSuccess) { cudaGetLastError(); return bail(CLBM_ERR_OOM); }
        if (cudaMemcpy(c->force, fb.data(), fb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(CLBM_ERR_CUDA);
    }

    // default state: f* of the rest equilibrium
    st = clbm_init_dev(c, nullptr, nullptr, nullptr);
    if (st == CLBM_OK) st = clbm_synchronize(c);
    if (st != CLBM_OK) return bail(st);
    *out = c;
    return CLBM_OK;
}

int clbm_init_dev(clbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    int st = check_ctx(c);
    if (st) return st;
    // the state lands in buf[0]: make_args(c, 1) writes its dst = buf[0]
    c->cur = 0;
    drop_graphs(c);
    if (c->format == CLBM_FP16 && !c->user_scale) {
        c->scale_k = 0;   // provisional pass at scale 1 to measure the deviations
        CLBM_CK(c, clbm::launch_init(make_args(c, 1), c->format, rho, ux, uy, c->stream));
        st = choose_scale(c);
        if (st) return st;
    }
    if (shan_chen(c))     // the force of the initial density
        CLBM_CK(c, clbm::launch_psi_prepare(make_args(c, 1), c->format, 0, rho, nullptr, c->psi, c->stream));
    CLBM_CK(c, clbm::launch_init(make_args(c, 1), c->format, rho, ux, uy, c->stream));
    return CLBM_OK;
}

int clbm_init(clbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    int st = check_ctx(c);
    if (st) return st;
    const size_t n = (size_t)c->nx * c->ny;
    // inputs that are all page-locked memory mapped into the device's
    // address space are read by the kernel in place, with no staging copy
    const double* m[3] = {mapped_host(const_cast<double*>(rho)), mapped_host(const_cast<double*>(ux)),
                          mapped_host(const_cast<double*>(uy))};
    if ((!rho || m[0]) && (!ux || m[1]) && (!uy || m[2])) {
        st = clbm_init_dev(c, m[0], m[1], m[2]);
        if (st) return st;
        return clbm_synchronize(c);
    }
    st = ensure_staging(c, 3 * n);
    if (st) return st;
    double* d[3] = {nullptr, nullptr, nullptr};
    const double* h[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k) {
        if (!h[k]) continue;
        d[k] = c->staging + k * n;
        CLBM_CK(c, cudaMemcpyAsync(d[k], h[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    st = clbm_init_dev(c, d[0], d[1], d[2]);
    if (st) return st;
    return clbm_synchronize(c);
}

int clbm_set_populations(clbm_ctx* c, const double* f, int pre_collision) {
    int st = check_ctx(c);
    if (st) return st;
    if (!f || (pre_collision != 0 && pre_collision != 1)) return CLBM_ERR_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    st = ensure_staging(c, 9 * n);
    if (st) return st;
    CLBM_CK(c, cudaMemcpyAsync(c->staging, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->cur = 0;
    drop_graphs(c);
    if (shan_chen(c) && pre_collision)    // the force of the state's density
        CLBM_CK(c, clbm::launch_psi_prepare(make_args(c, 1), c->format, 1, nullptr, c->staging, c->psi,
                                            c->stream));
    CLBM_CK(c, clbm::launch_set_populations(make_args(c, 1), c->format, c->staging, pre_collision, c->stream));
    return clbm_synchronize(c);
}

int clbm_get_populations(clbm_ctx* c, double* f, int pre_collision) {
    int st = check_ctx(c);
    if (st) return st;
    if (!f || (pre_collision != 0 && pre_collision != 1)) return CLBM_ERR_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    st = ensure_staging(c, 9 * n);
    if (st) return st;
    CLBM_CK(c, clbm::launch_get_populations(make_args(c, c->cur), c->format, c->staging, pre_collision,
                                            c->stream));
    CLBM_CK(c, cudaMemcpyAsync(f, c->staging, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return clbm_synchronize(c);
}

int clbm_get_window_async(clbm_ctx* c, int x0, int y0, int w, int h, double* f) {
    int st = check_ctx(c);
    if (st) return st;
    if (!f || w < 1 || h < 1 || x0 < 0 || y0 < 0 || x0 >= c->nx || y0 >= c->ny) return CLBM_ERR_ARG;
    const size_t n = (size_t)w * h;
    // page-locked host memory mapped into the device's address space: the
    // readout kernel writes it directly, with no copy-engine transfer between
    // the steps in the stream
    if (double* m = mapped_host(f)) {
        CLBM_CK(c, clbm::launch_window(make_args(c, c->cur), c->format, x0, y0, w, h, m, c->stream));
        return CLBM_OK;
    }
    st = ensure_staging(c, 9 * n);
    if (st) return st;
    CLBM_CK(c, clbm::launch_window(make_args(c, c->cur), c->format, x0, y0, w, h, c->staging, c->stream));
    CLBM_CK(c, cudaMemcpyAsync(f, c->staging, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return CLBM_OK;
}

int clbm_get_window(clbm_ctx* c, int x0, int y0, int w, int h, double* f) {
    int st = clbm_get_window_async(c, x0, y0, w, h, f);
    if (st) return st;
    return clbm_synchronize(c);
}

int clbm_step(clbm_ctx* c, int n) {
    int st = check_ctx(c);
    if (st) return st;
    if (n < 0) return CLBM_ERR_ARG;
    while (n > 0) {
        if (n >= kGraphSteps) {
            if (!c->graph[c->cur]) {
                st = build_graph(c, c->cur);
                if (st) return st;
            }
            CLBM_CK(c, cudaGraphLaunch(c->graph[c->cur], c->stream));
            n -= kGraphSteps;
        } else {
            CLBM_CK(c, launch_one_step(c, c->cur, c->stream));
            c->cur ^= 1;
            --n;
        }
    }
    return CLBM_OK;
}

int clbm_moments_dev(clbm_ctx* c, double* rho, double* ux, double* uy) {
    int st = check_ctx(c);
    if (st) return st;
    if ((st = psi_of_current(c))) return st;
    CLBM_CK(c, clbm::launch_moments(make_args(c, c->cur), c->format, rho, ux, uy, c->stream));
    return CLBM_OK;
}

int clbm_moments(clbm_ctx* c, double* rho, double* ux, double* uy) {
    int st = check_ctx(c);
    if (st) return st;
    const size_t n = (size_t)c->nx * c->ny;
    // outputs that are all mapped page-locked memory are written by the
    // kernel directly, without a device copy and a copy-engine transfer
    double* m[3] = {mapped_host(rho), mapped_host(ux), mapped_host(uy)};
    if ((!rho || m[0]) && (!ux || m[1]) && (!uy || m[2])) {
        if ((st = psi_of_current(c))) return st;
        CLBM_CK(c, clbm::launch_moments(make_args(c, c->cur), c->format, m[0], m[1], m[2], c->stream));
        return clbm_synchronize(c);
    }
    st = ensure_staging(c, 3 * n);
    if (st) return st;
    double* d[3] = {rho ? c->staging : nullptr, ux ? c->staging + n : nullptr,
                    uy ? c->staging + 2 * n : nullptr};
    if ((st = psi_of_current(c))) return st;
    CLBM_CK(c, clbm::launch_moments(make_args(c, c->cur), c->format, d[0], d[1], d[2], c->stream));
    double* h[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k)
        if (h[k])
            CLBM_CK(c, cudaMemcpyAsync(h[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return clbm_synchronize(c);
}

int clbm_reduce(clbm_ctx* c, double out[3]) {
    int st = check_ctx(c);
    if (st) return st;
    if (!out) return CLBM_ERR_ARG;
    double h[4];
    if ((st = psi_of_current(c))) return st;
    CLBM_CK(c, clbm::launch_reduce_moments(make_args(c, c->cur), c->format, c->partials, c->red_out, c->stream));
    CLBM_CK(c, cudaMemcpyAsync(h, c->red_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    st = clbm_synchronize(c);
    if (st) return st;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    if (h[3] != 0.0 || !clbm::all_finite(h, 3)) return CLBM_ERR_DIVERGED;
    return CLBM_OK;
}

int clbm_l2_error(clbm_ctx* c, const double* ua, const double* va, double* out) {
    int st = check_ctx(c);
    if (st) return st;
    if (!ua || !va || !out) return CLBM_ERR_ARG;
    const size_t n = (size_t)c->nx * c->ny;
    st = ensure_staging(c, 2 * n);
    if (st) return st;
    CLBM_CK(c, cudaMemcpyAsync(c->staging, ua, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CLBM_CK(c, cudaMemcpyAsync(c->staging + n, va, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    double h[4];
    if ((st = psi_of_current(c))) return st;
    CLBM_CK(c, clbm::launch_reduce_l2(make_args(c, c->cur), c->format, c->staging, c->staging + n,
                                      c->partials, c->red_out, c->stream));
    CLBM_CK(c, cudaMemcpyAsync(h, c->red_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    st = clbm_synchronize(c);
    if (st) return st;
    if (h[3] != 0.0 || !clbm::all_finite(h, 2)) return CLBM_ERR_DIVERGED;
    *out = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return CLBM_OK;
}

int clbm_set_forcing_scheme(clbm_ctx* c, int scheme) {
    int st = check_ctx(c);
    if (st) return st;
    if (scheme < CLBM_FORCING_CONSISTENT || scheme > CLBM_FORCING_M2) return CLBM_ERR_ARG;
    clbm::relax_constants(c->rates, scheme, c->relax);
    drop_graphs(c);
    return CLBM_OK;
}

int clbm_synchronize(clbm_ctx* c) {
    if (!c) return CLBM_ERR_ARG;
    if (c->sticky != CLBM_OK) return CLBM_ERR_STATE;
    CLBM_CK(c, cudaStreamSynchronize(c->stream));
    CLBM_CK(c, cudaGetLastError());
    return CLBM_OK;
}

int clbm_scale_exponent(const clbm_ctx* c) { return c ? c->scale_k : 0; }

int clbm_set_scale_exponent(clbm_ctx* c, int k) {
    int st = check_ctx(c);
    if (st) return st;
    if (k < 0 || k > 40 || (c->format != CLBM_FP16 && k != 0)) return CLBM_ERR_ARG;
    c->scale_k = k;
    c->user_scale = true;
    drop_graphs(c);
    return CLBM_OK;
}

int clbm_set_tuning(clbm_ctx* c, int vec_bytes, int packed, int prefetch, int stages) {
    int st = check_ctx(c);
    if (st) return st;
    if (vec_bytes != 8 && vec_bytes != 16) return CLBM_ERR_ARG;
    if (c->format == CLBM_FP64 && vec_bytes != 16) return CLBM_ERR_ARG;
    if (packed != 0 && packed != 1) return CLBM_ERR_ARG;
    if (prefetch < 0 || prefetch > 4) return CLBM_ERR_ARG;
    if (stages != 0 && stages != 2 && stages != 3) return CLBM_ERR_ARG;
    c->vec_bytes = vec_bytes;
    c->packed = c->format == CLBM_FP64 ? 0 : packed;
    c->prefetch = prefetch;
    c->stages = stages;
    drop_graphs(c);
    return build_vlist(c);        // the list depends on the vector width
}

int clbm_set_sparse(clbm_ctx* c, int mode) {
    int st = check_ctx(c);
    if (st) return st;
    if (mode != CLBM_SPARSE_OFF && mode != CLBM_SPARSE_ON && mode != CLBM_SPARSE_AUTO) return CLBM_ERR_ARG;
    c->sparse_mode = mode;
    drop_graphs(c);
    return build_vlist(c);
}

int clbm_sparse_tasks(const clbm_ctx* c) { return c ? c->vtasks : 0; }

int clbm_set_rounding(clbm_ctx* c, int mode) {
    int st = check_ctx(c);
    if (st) return st;
    if (mode != CLBM_ROUND_NEAREST && mode != CLBM_ROUND_STOCHASTIC) return CLBM_ERR_ARG;
    if (mode == CLBM_ROUND_STOCHASTIC && c->format != CLBM_FP16 && c->format != CLBM_BF16) return CLBM_ERR_ARG;
    if (mode == CLBM_ROUND_STOCHASTIC && !c->sr_step) {
        CLBM_CK(c, clbm::dev_alloc(&c->sr_step, sizeof(uint32_t)));
        CLBM_CK(c, cudaMemsetAsync(c->sr_step, 0, sizeof(uint32_t), c->stream));
        CLBM_CK(c, cudaStreamSynchronize(c->stream));
    }
    c->rounding = mode;
    drop_graphs(c);
    return CLBM_OK;
}

int clbm_get_tuning(const clbm_ctx* c, int* vec_bytes, int* packed, int* prefetch, int* stages) {
    if (!c) return CLBM_ERR_ARG;
    if (vec_bytes) *vec_bytes = c->vec_bytes;
    if (packed) *packed = c->packed;
    if (prefetch) *prefetch = c->prefetch;
    if (stages) *stages = c->stages;
    return CLBM_OK;
}

double clbm_bytes_per_update(const clbm_ctx* c) {
    if (!c) return 0.0;
    const double e = clbm::element_size(c->format);
    if (c->force_kind == CLBM_FORCE_SHAN_CHEN) {
        // + the psi pass (9 populations read, psi written) + psi read by the step
        const double cs = c->format == CLBM_FP64 ? 8.0 : 4.0;
        return 27.0 * e + 2.0 * cs;
    }
    return 18.0 * e + (c->lmask ? 1.125 : 0.0);
}

long long clbm_fluid_nodes(const clbm_ctx* c) { return c ? c->fluid : 0; }

int clbm_get_size(const clbm_ctx* c, int* nx, int* ny) {
    if (!c) return CLBM_ERR_ARG;
    if (nx) *nx = c->nx;
    if (ny) *ny = c->ny;
    return CLBM_OK;
}

int clbm_debug_fail_next(int what) {
    if (what != CLBM_FAIL_NONE && what != CLBM_FAIL_ALLOC && what != CLBM_FAIL_LAUNCH) return CLBM_ERR_ARG;
    clbm::g_fail_next.store(what);
    return CLBM_OK;
}

}  // extern "C"
