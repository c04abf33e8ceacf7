// clbm_batch.cu -- the batch C ABI of include/clbm.h: many independent
// lattices (uneven sizes, rates, forces, walls) advanced together, one fused
// step launch per time step over all of them, replayed from CUDA graphs, with
// an autotuner that picks the launch shape by timing it on the batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_device.cuh"
#include "clbm_host.h"
#include "clbm_internal.h"

using clbm::BatchDomain;
using clbm::BatchLaunch;
using clbm::StepArgs;

namespace {

const int kBatchGraphSteps = 32;   // even: a replay keeps the buffer parity

struct HostDomain {
    int nx, ny, pitch;
    size_t pop_off;        // byte offset of the domain's planes in each copy
    size_t mask_off, sbit_off;   // byte offsets in the mask allocation
    size_t force_off;      // byte offset in the force allocation
    bool has_mask;
    long long fluid;
    int scale_k;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

std::mutex g_tune_mutex;
struct Shape {
    int vec_bytes, packed, stages, schedule;
    int persist, resident, order;          // clbm_batch_set_mode
};
std::map<std::string, Shape> g_tune_cache;   // signature -> launch shape

// The autotuner's file cache: CLBM_TUNE_CACHE if set (empty: none), else
// $XDG_CACHE_HOME/clbm-batch-tuning.txt or ~/.cache/clbm-batch-tuning.txt.
std::string tune_file() {
    if (const char* e = std::getenv("CLBM_TUNE_CACHE")) return std::string(e);
    if (const char* x = std::getenv("XDG_CACHE_HOME")) return std::string(x) + "/clbm-batch-tuning.txt";
    if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/clbm-batch-tuning.txt";
    return std::string();
}

// One line per batch signature: the signature (no blanks), then the seven
// integers of its shape.
bool file_lookup(const std::string& key, Shape& out) {
    const std::string path = tune_file();
    if (path.empty()) return false;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string k;
        Shape s{};
        if ((ls >> k >> s.vec_bytes >> s.packed >> s.stages >> s.schedule >> s.persist >> s.resident >> s.order) &&
            k == key) {
            out = s;
            return true;
        }
    }
    return false;
}

void file_store(const std::string& key, const Shape& s) {
    const std::string path = tune_file();
    if (path.empty()) return;
    std::vector<std::string> keep;
    {
        std::ifstream in(path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            if ((ls >> k) && k != key) keep.push_back(line);
        }
    }
    std::ostringstream row;
    row << key << ' ' << s.vec_bytes << ' ' << s.packed << ' ' << s.stages << ' ' << s.schedule << ' '
        << s.persist << ' ' << s.resident << ' ' << s.order;
    keep.push_back(row.str());
    const std::string tmp = path + ".tmp";
    {
        std::ofstream out(tmp, std::ios::trunc);
        if (!out) return;                     // no writable cache: keep the in-process one only
        for (const auto& l : keep) out << l << '\n';
    }
    std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

struct clbm_batch {
    int count = 0, format = 0;
    std::vector<HostDomain> hd;
    std::vector<BatchDomain> doms;        // host copy of the descriptors
    std::vector<int> task0;
    long long ntasks = 0, fluid = 0;
    double bytes_per_step = 0.0;
    unsigned char* bufA = nullptr;
    unsigned char* bufB = nullptr;
    unsigned char* masks = nullptr;
    unsigned char* forces = nullptr;
    BatchDomain* d_doms = nullptr;
    int* d_task0 = nullptr;
    int parity = 0;                       // 0: current state in copy A
    int vec_bytes = 16, packed = 0, stages = 0, schedule = 1;
    int persist = 0, resident = 0, order = 0;   // clbm_batch_set_mode
    int nstream = 0, nres = 0;            // lattices streamed / held in shared memory
    std::vector<int> dev_order;           // device descriptor k: lattice dev_order[k]
    bool guo = false;                     // some lattice uses the M2 forcing scheme
    unsigned* d_done = nullptr;           // per-lattice counters of persistent launches
    int* d_status = nullptr;              // 1 once a wait of a persistent launch gave up
    int* d_res_first = nullptr;           // resident lattices of each resident block
    int res_blocks = 0;
    unsigned spin_limit = 1u << 20, delay_ns = 0u;
    bool graphs_off = false;              // capture of the launch not available
    bool ran_persist = false;             // a persistent launch was issued
    cudaStream_t stream = nullptr, cap = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double* staging = nullptr;
    size_t staging_cap = 0;
    double* partials = nullptr;
    double* red_out = nullptr;
    int sticky = CLBM_OK;
};

namespace {

int cuda_status(clbm_batch* b, cudaError_t e) {
    if (e == cudaSuccess) return CLBM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return CLBM_ERR_OOM;
    }
    if (b) b->sticky = CLBM_ERR_CUDA;
    return CLBM_ERR_CUDA;
}

#define BATCH_CK(b, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_status(b, e_);  \
    } while (0)

int check_batch(clbm_batch* b) {
    if (!b) return CLBM_ERR_ARG;
    if (b->sticky != CLBM_OK) return CLBM_ERR_STATE;
    return CLBM_OK;
}

void drop_graphs(clbm_batch* b) {
    for (auto& g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Descriptors and the flat task list for the current launch shape, in the
// launch order: the streamed lattices (as given, or the largest first), then
// those held in shared memory by persistent launches (the smallest ones
// whose state fits twice in a block's stage memory, at most one per eight
// blocks' worth of the batch and never all of it).
int upload_descriptors(clbm_batch* b) {
    const int V = clbm::vector_width_of(b->format, b->vec_bytes);
    std::vector<int> stream_ids, res_ids;
    std::vector<int> ids(b->count);
    for (int d = 0; d < b->count; ++d) ids[d] = d;
    if (b->persist && b->resident) {
        int mm = 0;
        for (const auto& h : b->hd) mm += h.has_mask;
        const int mask_mode = mm == 0 ? 0 : mm == b->count ? 1 : 2;
        const size_t room = clbm::batch_stage_bytes(b->format, b->vec_bytes, b->stages, mask_mode);
        const size_t esz = (size_t)clbm::element_size(b->format);
        std::vector<int> by_size = ids;
        std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) {
            return (long long)b->hd[x].nx * b->hd[x].ny < (long long)b->hd[y].nx * b->hd[y].ny;
        });
        for (int d : by_size) {
            const size_t need = 2 * 9 * (size_t)b->hd[d].nx * b->hd[d].ny * esz;
            if (need > room || (int)res_ids.size() >= 128 || (int)res_ids.size() + 1 >= b->count) break;
            res_ids.push_back(d);
        }
    }
    std::vector<bool> is_res(b->count, false);
    for (int d : res_ids) is_res[d] = true;
    for (int d : ids)
        if (!is_res[d]) stream_ids.push_back(d);
    if (b->order == 1)
        std::stable_sort(stream_ids.begin(), stream_ids.end(), [&](int x, int y) {
            return b->hd[x].fluid > b->hd[y].fluid;
        });
    b->dev_order = stream_ids;
    b->dev_order.insert(b->dev_order.end(), res_ids.begin(), res_ids.end());
    b->nstream = (int)stream_ids.size();
    b->nres = (int)res_ids.size();
    for (int d = 0; d < b->count; ++d) {
        StepArgs& a = b->doms[d].a;
        a.vec_bytes = b->vec_bytes;
        a.packed = b->packed;
        a.prefetch = 0;
        a.stages = 0;
        // flat tasks: 32 consecutive vectors of the lattice in row-major
        // vector order, so a ragged row end shares its task with the next row
        a.chunks = (a.geo.nx + V - 1) / V;
        a.ntasks = ((long long)a.geo.ny * a.chunks + 31) / 32;
        const double sc = std::ldexp(1.0, b->hd[d].scale_k);
        a.scale = sc;
        a.inv_scale = 1.0 / sc;
        clbm::derive_args(a);
    }
    // the flat task list over the streamed lattices, in the launch order
    std::vector<BatchDomain> dev(b->count);
    long long t = 0;
    for (int k = 0; k < b->count; ++k) {
        dev[k] = b->doms[b->dev_order[k]];
        b->task0[k] = (int)t;
        if (k < b->nstream) t += dev[k].a.ntasks;
    }
    b->ntasks = t;
    // resident lattices packed onto few blocks (they are small): a block
    // takes lattices until its nodes reach a quarter of the streamed nodes
    // per block of a GB300-sized grid (152 SMs x 4 blocks), since a block
    // steps them one node per thread
    std::vector<int> rf(1, 0);
    if (b->nres > 0) {
        long long streamed = 0;
        for (int k = 0; k < b->nstream; ++k) streamed += (long long)dev[k].a.geo.nx * dev[k].a.geo.ny;
        const long long cap = streamed / (4 * 608) + 1;
        long long acc = 0;
        for (int r = 0; r < b->nres; ++r) {
            const long long nodes = (long long)dev[b->nstream + r].a.geo.nx * dev[b->nstream + r].a.geo.ny;
            if (acc > 0 && acc + nodes > cap) {
                rf.push_back(r);
                acc = 0;
            }
            acc += nodes;
        }
        rf.push_back(b->nres);
    }
    b->res_blocks = (int)rf.size() - 1;
    BATCH_CK(b, cudaMemcpyAsync(b->d_res_first, rf.data(), rf.size() * sizeof(int), cudaMemcpyHostToDevice,
                                b->stream));
    BATCH_CK(b, cudaMemcpyAsync(b->d_doms, dev.data(), dev.size() * sizeof(BatchDomain),
                                cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, cudaMemcpyAsync(b->d_task0, b->task0.data(), b->task0.size() * sizeof(int),
                                cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    return CLBM_OK;
}

BatchLaunch launch_args(const clbm_batch* b, int parity) {
    BatchLaunch l{};
    l.doms = b->d_doms;
    l.task0 = b->d_task0;
    l.ndom = b->count;
    l.ntasks = (int)b->ntasks;
    l.parity = parity;
    l.vec_bytes = b->vec_bytes;
    l.packed = b->packed;
    l.stages = b->stages;
    l.schedule = b->schedule;
    l.guo = 0;
    int masked = 0;
    for (const auto& d : b->doms) {
        if (d.a.relax.d[9] != 0.0) l.guo = 1;
        masked += d.a.lmask != nullptr;
    }
    l.mask_mode = masked == 0 ? 0 : masked == b->count ? 1 : 2;
    l.ndom = b->nstream;
    l.persist = b->persist;
    l.nsteps = 1;
    l.nres = b->nres;
    l.res_blocks = b->res_blocks;
    l.res_first = b->d_res_first;
    l.done = b->d_done;
    l.status = b->d_status;
    l.spin_limit = b->spin_limit;
    l.delay_ns = b->delay_ns;
    return l;
}

// Launch n steps from parity p: one persistent launch, or n step launches.
cudaError_t launch_steps(const clbm_batch* b, int p, int n, cudaStream_t s) {
    if (b->persist) {
        BatchLaunch l = launch_args(b, p);
        l.nsteps = n;
        return clbm::launch_batch_step(l, b->format, s);
    }
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < n && err == cudaSuccess; ++k) {
        err = clbm::launch_batch_step(launch_args(b, p), b->format, s);
        p ^= 1;
    }
    return err;
}

// StepArgs of domain d whose src and dst are both its current copy (for the
// per-node helper kernels, which read src or write dst).
StepArgs current_args(const clbm_batch* b, int d) {
    StepArgs a = b->doms[d].a;
    void* cur = b->parity ? a.dst : const_cast<void*>(a.src);
    a.src = cur;
    a.dst = cur;
    return a;
}

int ensure_staging(clbm_batch* b, size_t doubles) {
    if (b->staging_cap >= doubles) return CLBM_OK;
    if (b->staging) cudaFree(b->staging);
    b->staging = nullptr;
    b->staging_cap = 0;
    BATCH_CK(b, clbm::dev_alloc(&b->staging, doubles * sizeof(double)));
    b->staging_cap = doubles;
    return CLBM_OK;
}

int build_graph(clbm_batch* b, int parity) {
    cudaGraph_t g = nullptr;
    BATCH_CK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = launch_steps(b, parity, kBatchGraphSteps, b->cap);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (err != cudaSuccess && b->persist) {
        // a cooperative launch that cannot be captured: launch it directly
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        b->graphs_off = true;
        return CLBM_OK;
    }
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(b, err);
    }
    BATCH_CK(b, e2);
    cudaError_t e3 = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    BATCH_CK(b, e3);
    return CLBM_OK;
}

int check_domain(const clbm_batch* b, int d) { return (d >= 0 && d < b->count) ? CLBM_OK : CLBM_ERR_ARG; }

std::string signature(const clbm_batch* b) {
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string s = std::string(prop.name) + "|" + std::to_string(b->format) + "|" +
                    std::to_string(b->count);
    unsigned long long h = 1469598103934665603ULL;   // FNV-1a over the shapes
    for (const auto& d : b->hd) {
        const unsigned long long v[3] = {(unsigned long long)d.nx, (unsigned long long)d.ny,
                                         (unsigned long long)d.has_mask};
        for (unsigned long long x : v) {
            h ^= x;
            h *= 1099511628211ULL;
        }
    }
    s += "|" + std::to_string(h);
    for (auto& ch : s)
        if (ch == ' ' || ch == '\t') ch = '_';
    return s;
}

}  // namespace

extern "C" {

int clbm_batch_destroy(clbm_batch* b) {
    if (!b) return CLBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    void* ptrs[] = {b->bufA, b->bufB, b->masks, b->forces, b->d_doms, b->d_task0, b->staging,
                    b->partials, b->red_out, b->d_done, b->d_status, b->d_res_first};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return CLBM_OK;
}

int clbm_batch_create(clbm_batch** out, int count, const clbm_domain_desc* d, int format,
                      void* stream) {
    if (!out) return CLBM_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !d) return CLBM_ERR_ARG;
    for (int k = 0; k < count; ++k) {
        const int st = clbm::check_lattice_args(d[k].nx, d[k].ny, d[k].rates, d[k].force_kind,
                                                d[k].force, d[k].fx, d[k].fy, format);
        if (st != CLBM_OK) return st;
        if (d[k].forcing < CLBM_FORCING_CONSISTENT || d[k].forcing > CLBM_FORCING_M2) return CLBM_ERR_ARG;
        if (d[k].force_kind == CLBM_FORCE_SHAN_CHEN) return CLBM_ERR_ARG;   // single lattices only
    }
    {   // the flat task list is indexed in 32 bits; its longest form has
        // 64-node chunks (8-byte vectors of 32-bit or 16-byte vectors of
        // 64-bit values)
        long long worst = 0;
        for (int k = 0; k < count; ++k) worst += (long long)d[k].ny * ((d[k].nx + 63) / 64);
        if (worst >= (1LL << 31)) return CLBM_ERR_ARG;
    }
    clbm_batch* b = new (std::nothrow) clbm_batch();
    if (!b) return CLBM_ERR_OOM;
    auto bail = [&](int s) { clbm_batch_destroy(b); return s; };
    b->count = count;
    b->format = format;
    if (format != CLBM_FP64) {
        b->packed = 1;
        b->stages = 2;
        b->schedule = CLBM_SCHEDULE_CONTIGUOUS;
    }
    b->hd.resize(count);
    b->doms.assign(count, BatchDomain{});
    b->task0.assign(count, 0);
    const int esz = clbm::element_size(format);
    const size_t fsz = format == CLBM_FP64 ? sizeof(double) : sizeof(float);

    // layout: populations, masks and forces of every domain in three
    // allocations (two population copies), each part on a 256-byte boundary
    size_t pop = 0, msk = 0, frc = 0;
    std::vector<std::vector<uint8_t>> lm(count), sb(count);
    for (int k = 0; k < count; ++k) {
        HostDomain& h = b->hd[k];
        h.nx = d[k].nx;
        h.ny = d[k].ny;
        h.pitch = clbm::row_pitch(h.nx, format);
        h.pop_off = pop;
        pop += align256((size_t)9 * h.pitch * h.ny * esz);
        long long nsolid = 0;
        if (d[k].solid) nsolid = clbm::build_solid_masks(d[k].solid, h.nx, h.ny, h.pitch, lm[k], sb[k]);
        h.has_mask = nsolid > 0;
        h.fluid = (long long)h.nx * h.ny - nsolid;
        if (h.has_mask) {
            h.mask_off = msk;
            msk += align256(lm[k].size());
            h.sbit_off = msk;
            msk += align256(sb[k].size());
        }
        h.force_off = frc;
        frc += align256(clbm::force_values(d[k].force_kind, h.nx, h.ny) * fsz);
        h.scale_k = 0;
        b->fluid += h.fluid;
        b->bytes_per_step += (double)h.fluid * (18.0 * esz + (h.has_mask ? 1.125 : 0.0));
    }

    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(CLBM_ERR_CUDA);
        b->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return bail(CLBM_ERR_CUDA);
    if (clbm::dev_alloc(&b->bufA, pop) != cudaSuccess || clbm::dev_alloc(&b->bufB, pop) != cudaSuccess ||
        (msk && clbm::dev_alloc(&b->masks, msk) != cudaSuccess) ||
        (frc && clbm::dev_alloc(&b->forces, frc) != cudaSuccess) ||
        clbm::dev_alloc(&b->d_doms, count * sizeof(BatchDomain)) != cudaSuccess ||
        clbm::dev_alloc(&b->d_task0, count * sizeof(int)) != cudaSuccess ||
        clbm::dev_alloc(&b->partials, (size_t)clbm::reduce_partials_count() * 4 * sizeof(double)) != cudaSuccess ||
        clbm::dev_alloc(&b->red_out, 4 * sizeof(double)) != cudaSuccess ||
        clbm::dev_alloc(&b->d_done, count * sizeof(unsigned)) != cudaSuccess ||
        clbm::dev_alloc(&b->d_status, sizeof(int)) != cudaSuccess ||
        clbm::dev_alloc(&b->d_res_first, (count + 1) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return bail(CLBM_ERR_OOM);
    }
    if (cudaMemsetAsync(b->bufA, 0, pop, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->bufB, 0, pop, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess)
        return bail(CLBM_ERR_CUDA);

    for (int k = 0; k < count; ++k) {
        HostDomain& h = b->hd[k];
        StepArgs& a = b->doms[k].a;
        a.src = b->bufA + h.pop_off;
        a.dst = b->bufB + h.pop_off;
        a.geo.nx = h.nx;
        a.geo.ny = h.ny;
        a.geo.pitch = h.pitch;
        a.geo.plane = (long long)h.pitch * h.ny;
        a.force_kind = d[k].force_kind;
        a.fx = d[k].fx;
        a.fy = d[k].fy;
        a.rho0 = 1.0;
        clbm::relax_constants(d[k].rates, d[k].forcing, a.relax);
        if (d[k].forcing == CLBM_FORCING_M2) b->guo = true;
        if (h.has_mask) {
            a.lmask = b->masks + h.mask_off;
            a.sbits = b->masks + h.sbit_off;
            clbm::plain_row_range(d[k].solid, h.nx, h.ny, a.plain_y0, a.plain_y1);
            if (cudaMemcpy(b->masks + h.mask_off, lm[k].data(), lm[k].size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(b->masks + h.sbit_off, sb[k].data(), sb[k].size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(CLBM_ERR_CUDA);
        }
        const size_t nf = clbm::force_values(d[k].force_kind, h.nx, h.ny);
        if (nf) {
            std::vector<unsigned char> fb;
            clbm::force_in_compute_type(d[k].force, nf, format, fb);
            a.force = b->forces + h.force_off;
            if (cudaMemcpy(b->forces + h.force_off, fb.data(), fb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(CLBM_ERR_CUDA);
        }
    }
    int st = upload_descriptors(b);
    if (st != CLBM_OK) return bail(st);
    for (int k = 0; k < count && st == CLBM_OK; ++k) st = clbm_batch_init(b, k, nullptr, nullptr, nullptr);
    if (st != CLBM_OK) return bail(st);
    *out = b;
    return CLBM_OK;
}

int clbm_batch_init(clbm_batch* b, int dom, const double* rho, const double* ux, const double* uy) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    const HostDomain& h = b->hd[dom];
    const size_t n = (size_t)h.nx * h.ny;
    st = ensure_staging(b, 3 * n);
    if (st) return st;
    double* dv[3] = {nullptr, nullptr, nullptr};
    const double* hv[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k) {
        if (!hv[k]) continue;
        dv[k] = b->staging + k * n;
        BATCH_CK(b, cudaMemcpyAsync(dv[k], hv[k], n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    }
    if (b->format == CLBM_FP16) {
        // provisional pass at scale 1, then the run scale from the deviations
        b->hd[dom].scale_k = 0;
        b->doms[dom].a.scale = b->doms[dom].a.inv_scale = 1.0;
        BATCH_CK(b, clbm::launch_init(current_args(b, dom), b->format, dv[0], dv[1], dv[2], b->stream));
        double mx = 0.0;
        BATCH_CK(b, cudaMemsetAsync(b->red_out, 0, sizeof(double), b->stream));
        BATCH_CK(b, clbm::launch_max_abs_dev(current_args(b, dom), b->format, b->red_out, b->stream));
        BATCH_CK(b, cudaMemcpyAsync(&mx, b->red_out, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BATCH_CK(b, cudaStreamSynchronize(b->stream));
        b->hd[dom].scale_k = clbm::fp16_scale_exponent(mx);
        st = upload_descriptors(b);
        if (st) return st;
    }
    BATCH_CK(b, clbm::launch_init(current_args(b, dom), b->format, dv[0], dv[1], dv[2], b->stream));
    return clbm_batch_synchronize(b);
}

int clbm_batch_set_populations(clbm_batch* b, int dom, const double* f, int pre_collision) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    if (!f || (pre_collision != 0 && pre_collision != 1)) return CLBM_ERR_ARG;
    const size_t n = (size_t)b->hd[dom].nx * b->hd[dom].ny;
    if ((st = ensure_staging(b, 9 * n))) return st;
    BATCH_CK(b, cudaMemcpyAsync(b->staging, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, clbm::launch_set_populations(current_args(b, dom), b->format, b->staging, pre_collision,
                                             b->stream));
    return clbm_batch_synchronize(b);
}

int clbm_batch_get_populations(clbm_batch* b, int dom, double* f, int pre_collision) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    if (!f || (pre_collision != 0 && pre_collision != 1)) return CLBM_ERR_ARG;
    const size_t n = (size_t)b->hd[dom].nx * b->hd[dom].ny;
    if ((st = ensure_staging(b, 9 * n))) return st;
    BATCH_CK(b, clbm::launch_get_populations(current_args(b, dom), b->format, b->staging, pre_collision,
                                             b->stream));
    BATCH_CK(b, cudaMemcpyAsync(f, b->staging, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return clbm_batch_synchronize(b);
}

int clbm_batch_step(clbm_batch* b, int n) {
    int st = check_batch(b);
    if (st) return st;
    if (n < 0) return CLBM_ERR_ARG;
    if (b->persist && n > 0) b->ran_persist = true;
    while (n > 0) {
        if (n >= kBatchGraphSteps && !b->graphs_off) {
            if (!b->graph[b->parity] && (st = build_graph(b, b->parity))) return st;
            if (b->graphs_off) continue;          // capture unavailable: launch directly
            BATCH_CK(b, cudaGraphLaunch(b->graph[b->parity], b->stream));
            n -= kBatchGraphSteps;
        } else {
            if (clbm::take_launch_failure()) return cuda_status(b, cudaErrorLaunchFailure);   // test hook
            // persistent: one launch for the rest (at most a graph's worth)
            const int m = b->persist ? (n < kBatchGraphSteps ? n : kBatchGraphSteps) : 1;
            BATCH_CK(b, launch_steps(b, b->parity, m, b->stream));
            if (m & 1) b->parity ^= 1;
            n -= m;
        }
    }
    return CLBM_OK;
}

int clbm_batch_moments(clbm_batch* b, int dom, double* rho, double* ux, double* uy) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    const size_t n = (size_t)b->hd[dom].nx * b->hd[dom].ny;
    if ((st = ensure_staging(b, 3 * n))) return st;
    double* dv[3] = {rho ? b->staging : nullptr, ux ? b->staging + n : nullptr,
                     uy ? b->staging + 2 * n : nullptr};
    BATCH_CK(b, clbm::launch_moments(current_args(b, dom), b->format, dv[0], dv[1], dv[2], b->stream));
    double* hv[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k)
        if (hv[k])
            BATCH_CK(b, cudaMemcpyAsync(hv[k], dv[k], n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return clbm_batch_synchronize(b);
}

int clbm_batch_reduce(clbm_batch* b, int dom, double out[3]) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    if (!out) return CLBM_ERR_ARG;
    double h[4];
    BATCH_CK(b, clbm::launch_reduce_moments(current_args(b, dom), b->format, b->partials, b->red_out, b->stream));
    BATCH_CK(b, cudaMemcpyAsync(h, b->red_out, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    if ((st = clbm_batch_synchronize(b))) return st;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    if (h[3] != 0.0 || !clbm::all_finite(h, 3)) return CLBM_ERR_DIVERGED;
    return CLBM_OK;
}

int clbm_batch_l2_error(clbm_batch* b, int dom, const double* ua, const double* va, double* out) {
    int st = check_batch(b);
    if (st) return st;
    if ((st = check_domain(b, dom))) return st;
    if (!ua || !va || !out) return CLBM_ERR_ARG;
    const size_t n = (size_t)b->hd[dom].nx * b->hd[dom].ny;
    if ((st = ensure_staging(b, 2 * n))) return st;
    BATCH_CK(b, cudaMemcpyAsync(b->staging, ua, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, cudaMemcpyAsync(b->staging + n, va, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    double h[4];
    BATCH_CK(b, clbm::launch_reduce_l2(current_args(b, dom), b->format, b->staging, b->staging + n,
                                       b->partials, b->red_out, b->stream));
    BATCH_CK(b, cudaMemcpyAsync(h, b->red_out, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    if ((st = clbm_batch_synchronize(b))) return st;
    if (h[3] != 0.0 || !clbm::all_finite(h, 2)) return CLBM_ERR_DIVERGED;
    *out = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return CLBM_OK;
}

int clbm_batch_set_tuning(clbm_batch* b, int vec_bytes, int packed, int stages, int schedule) {
    int st = check_batch(b);
    if (st) return st;
    if (vec_bytes != 8 && vec_bytes != 16) return CLBM_ERR_ARG;
    if (packed != 0 && packed != 1) return CLBM_ERR_ARG;
    if (stages != 0 && stages != 2 && stages != 3) return CLBM_ERR_ARG;
    if (schedule != CLBM_SCHEDULE_CONTIGUOUS && schedule != CLBM_SCHEDULE_INTERLEAVED) return CLBM_ERR_ARG;
    if (b->format == CLBM_FP64 && (vec_bytes != 16 || packed != 0)) return CLBM_ERR_ARG;
    if (b->persist && stages == 0) return CLBM_ERR_ARG;          // persistent launches are staged
    b->vec_bytes = vec_bytes;
    b->packed = packed;
    b->stages = stages;
    b->schedule = schedule;
    return upload_descriptors(b);
}

int clbm_batch_get_tuning(const clbm_batch* b, int* vec_bytes, int* packed, int* stages,
                          int* schedule) {
    if (!b) return CLBM_ERR_ARG;
    if (vec_bytes) *vec_bytes = b->vec_bytes;
    if (packed) *packed = b->packed;
    if (stages) *stages = b->stages;
    if (schedule) *schedule = b->schedule;
    return CLBM_OK;
}

// The launch shape and mode of a tuning candidate.
int apply_shape(clbm_batch* b, const Shape& c) {
    int st;
    if (b->persist && (st = clbm_batch_set_mode(b, 0, 0, 0))) return st;
    if ((st = clbm_batch_set_tuning(b, c.vec_bytes, c.packed, c.stages, c.schedule))) return st;
    return clbm_batch_set_mode(b, c.persist, c.resident, c.order);
}

int clbm_batch_autotune(clbm_batch* b, int steps, double* ms_per_step) {
    int st = check_batch(b);
    if (st) return st;
    if (steps < 1) return CLBM_ERR_ARG;
    const std::string key = signature(b);
    if (!ms_per_step) {
        Shape c{};
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                c = it->second;
                hit = true;
            } else if (file_lookup(key, c)) {
                g_tune_cache[key] = c;
                hit = true;
            }
        }
        if (hit) return apply_shape(b, c);
    }
    cudaEvent_t e0, e1;
    BATCH_CK(b, cudaEventCreate(&e0));
    BATCH_CK(b, cudaEventCreate(&e1));
    double best = 1e300;
    Shape pick{};
    auto time_shape = [&](const Shape& c) -> int {
        int s2 = apply_shape(b, c);
        if (s2) return s2;
        if ((s2 = clbm_batch_step(b, 2))) return s2;                 // warm-up
        cudaEventRecord(e0, b->stream);
        if ((s2 = clbm_batch_step(b, steps))) return s2;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_status(b, cudaGetLastError());
        if ((s2 = clbm_batch_synchronize(b))) return s2;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / steps < best) {
            best = ms / steps;
            pick = c;
        }
        return CLBM_OK;
    };
    // 1: vector width x packing x ring depth x schedule, one launch per step
    for (int sch : {CLBM_SCHEDULE_INTERLEAVED, CLBM_SCHEDULE_CONTIGUOUS}) {
        for (int stg : {2, 3, 0}) {
            if (b->format == CLBM_FP64) {
                if (!st) st = time_shape({16, 0, stg, sch, 0, 0, 0});
            } else {
                for (int v : {16, 8})
                    for (int p : {1, 0})
                        if (!st) st = time_shape({v, p, stg, sch, 0, 0, 0});
            }
        }
    }
    // 2: around the best of those, the lattice order and persistent launches
    // (ring depth x small lattices in shared memory x order)
    if (!st) {
        const Shape base = pick;
        st = time_shape({base.vec_bytes, base.packed, base.stages, base.schedule, 0, 0, 1});
        if (!b->guo)
            for (int stg : {2, 3})
                for (int res : {0, 1})
                    for (int ord : {0, 1})
                        if (!st) st = time_shape({base.vec_bytes, base.packed, stg, CLBM_SCHEDULE_CONTIGUOUS, 1, res, ord});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = pick;
        file_store(key, pick);
    }
    if (ms_per_step) *ms_per_step = best;
    return apply_shape(b, pick);
}

int clbm_batch_synchronize(clbm_batch* b) {
    if (!b) return CLBM_ERR_ARG;
    if (b->sticky != CLBM_OK) return CLBM_ERR_STATE;
    BATCH_CK(b, cudaStreamSynchronize(b->stream));
    BATCH_CK(b, cudaGetLastError());
    if (b->ran_persist) {
        int h = 0;     // did a wait of a persistent launch give up?
        BATCH_CK(b, cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (h != 0) {
            b->sticky = CLBM_ERR_TIMEOUT;
            return CLBM_ERR_TIMEOUT;
        }
    }
    return CLBM_OK;
}

int clbm_batch_set_mode(clbm_batch* b, int persistent, int resident, int order) {
    int st = check_batch(b);
    if (st) return st;
    if ((persistent != 0 && persistent != 1) || (resident != 0 && resident != 1) || (order != 0 && order != 1))
        return CLBM_ERR_ARG;
    if (persistent && (b->stages == 0 || b->guo)) return CLBM_ERR_ARG;
    if (resident && !persistent) return CLBM_ERR_ARG;
    b->persist = persistent;
    b->resident = resident;
    b->order = order;
    b->graphs_off = false;
    return upload_descriptors(b);
}

int clbm_batch_get_mode(const clbm_batch* b, int* persistent, int* resident, int* order) {
    if (!b) return CLBM_ERR_ARG;
    if (persistent) *persistent = b->persist;
    if (resident) *resident = b->resident;
    if (order) *order = b->order;
    return CLBM_OK;
}

int clbm_batch_resident_lattices(const clbm_batch* b) { return b ? b->nres : 0; }

int clbm_batch_set_wait(clbm_batch* b, long long spin_limit, long long delay_ns) {
    int st = check_batch(b);
    if (st) return st;
    if (spin_limit < 0 || spin_limit > 0xffffffffLL || delay_ns < 0 || delay_ns > 100000000LL) return CLBM_ERR_ARG;
    b->spin_limit = (unsigned)spin_limit;
    b->delay_ns = (unsigned)delay_ns;
    drop_graphs(b);
    return CLBM_OK;
}

long long clbm_batch_fluid_nodes(const clbm_batch* b) { return b ? b->fluid : 0; }

double clbm_batch_bytes_per_step(const clbm_batch* b) { return b ? b->bytes_per_step : 0.0; }

int clbm_batch_scale_exponent(const clbm_batch* b, int dom) {
    return (b && dom >= 0 && dom < b->count) ? b->hd[dom].scale_k : 0;
}

}  // extern "C"
