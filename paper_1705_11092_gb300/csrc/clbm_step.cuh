// clbm_step.cuh -- the fused pull-stream + collide + force kernel of one
// D2Q9 cascaded LBM time step (Fei & Luo, arXiv:1705.11092, Eq. 9-15 and the
// halfway bounce-back of Sec. 4A), templated on the storage format and the
// launch shape; instantiated once per format by clbm_step_<format>.cu.
//
// Layout in HBM: 9 population planes [i][y][x] (structure of arrays), rows
// padded to 128 bytes, two copies (ping-pong).  Each warp owns 32 * V
// consecutive nodes of one row; each lane moves one 16- or 8-byte vector per
// plane, so every plane access is one coalesced warp transaction.  Pull
// streaming reads plane i from the node x - e_i: the row offset is a
// different row base, the +-1 column offset is one element shifted in from
// the neighbouring lane (warp shuffle), with a separate element fetch at the
// warp edges and at the periodic wrap.
#pragma once

#include <type_traits>

#include "clbm_device.cuh"
#include "clbm_internal.h"

namespace clbm {

// ---------------------------------------------------------------------------
// raw element access inside a thread's vector held as NW 32-bit words
// ---------------------------------------------------------------------------
template <class S> struct Raw {
    using E = uint32_t;   // 16-bit and 32-bit elements travel as one word
};
template <> struct Raw<double> {
    using E = unsigned long long;
};

template <class S, int NW>
__device__ __forceinline__ typename Raw<S>::E raw_get(const uint32_t (&w)[NW], int j) {
    if constexpr (sizeof(S) == 8) {
        return ((unsigned long long)w[2 * j + 1] << 32) | w[2 * j];
    } else if constexpr (sizeof(S) == 4) {
        return w[j];
    } else {
        return (w[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
    }
}

template <class S, int NW>
__device__ __forceinline__ void raw_set(uint32_t (&w)[NW], int j, typename Raw<S>::E v) {
    if constexpr (sizeof(S) == 8) {
        w[2 * j] = (uint32_t)v;
        w[2 * j + 1] = (uint32_t)(v >> 32);
    } else if constexpr (sizeof(S) == 4) {
        w[j] = v;
    } else {
        w[j >> 1] = (j & 1) ? ((w[j >> 1] & 0x0000ffffu) | (v << 16))
                            : ((w[j >> 1] & 0xffff0000u) | (v & 0xffffu));
    }
}

// w <- o at the nodes whose link bounces, by whole-word bit selects: byte j
// of lb holds node j's link in bit 0 (the link word shifted right by i - 1
// for plane i); nodes without the link keep w.
template <class S, int NW>
__device__ __forceinline__ void link_select(uint32_t (&w)[NW], const uint32_t (&o)[NW],
                                            unsigned long long lb) {
    const unsigned long long bm = (lb & 0x0101010101010101ull) * 0xffull;   // byte j: 0xff or 0
    const uint32_t lo = (uint32_t)bm, hi = (uint32_t)(bm >> 32);
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        uint32_t m;
        if constexpr (sizeof(S) == 8) {          // words 2j, 2j+1: node j
            const int j = k >> 1;
            m = __byte_perm(j < 4 ? lo : hi, 0u, (j & 3) * 0x1111);
        } else if constexpr (sizeof(S) == 4) {   // word k: node k
            m = __byte_perm(k < 4 ? lo : hi, 0u, (k & 3) * 0x1111);
        } else {                                 // word k: nodes 2k (low half), 2k+1
            const int j = 2 * k;
            m = __byte_perm(j < 4 ? lo : hi, 0u, (j & 3) * 0x0011 + ((j + 1) & 3) * 0x1100);
        }
        w[k] = (w[k] & ~m) | (o[k] & m);
    }
}

// element j <- element j-1, element 0 <- L   (source at x - 1)
template <class S, int NW>
__device__ __forceinline__ void shift_in_left(uint32_t (&w)[NW], typename Raw<S>::E L) {
    if constexpr (sizeof(S) == 2) {
        // __byte_perm(a, b, 0x5432) = high half of a | low half of b << 16
#pragma unroll
        for (int k = NW - 1; k > 0; --k) w[k] = __byte_perm(w[k - 1], w[k], 0x5432);
        w[0] = __byte_perm(L << 16, w[0], 0x5432);
    } else {
        constexpr int V = NW * 4 / sizeof(S);
#pragma unroll
        for (int j = V - 1; j > 0; --j) raw_set<S, NW>(w, j, raw_get<S, NW>(w, j - 1));
        raw_set<S, NW>(w, 0, L);
    }
}

// element j <- element j+1, element V-1 <- R   (source at x + 1)
template <class S, int NW>
__device__ __forceinline__ void shift_in_right(uint32_t (&w)[NW], typename Raw<S>::E R) {
    if constexpr (sizeof(S) == 2) {
#pragma unroll
        for (int k = 0; k < NW - 1; ++k) w[k] = __byte_perm(w[k], w[k + 1], 0x5432);
        w[NW - 1] = __byte_perm(w[NW - 1], R, 0x5432);
    } else {
        constexpr int V = NW * 4 / sizeof(S);
#pragma unroll
        for (int j = 0; j < V - 1; ++j) raw_set<S, NW>(w, j, raw_get<S, NW>(w, j + 1));
        raw_set<S, NW>(w, V - 1, R);
    }
}

template <int NW>
__device__ __forceinline__ void ld_vec(const void* p, uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    }
}

template <int NW>
__device__ __forceinline__ void st_vec(void* p, const uint32_t (&w)[NW]) {
    if constexpr (NW == 4) {
        __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
    } else {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
    }
}

template <class S>
__device__ __forceinline__ typename Raw<S>::E ld_elem(const S* p) {
    if constexpr (sizeof(S) == 8) {
        return __ldg(reinterpret_cast<const unsigned long long*>(p));
    } else if constexpr (sizeof(S) == 4) {
        return __ldg(reinterpret_cast<const unsigned int*>(p));
    } else {
        return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p));
    }
}

// element j of a vector as the compute type (FP64, FP32 words; no scaling)
template <class S, int NW>
__device__ __forceinline__ typename Fmt<S>::C elem_get(const uint32_t (&w)[NW], int j) {
    if constexpr (sizeof(S) == 8) {
        return __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]);
    } else {
        return __uint_as_float(w[j]);
    }
}

template <class S, int NW>
__device__ __forceinline__ void elem_set(uint32_t (&w)[NW], int j, typename Fmt<S>::C v) {
    if constexpr (sizeof(S) == 8) {
        w[2 * j] = (uint32_t)__double2loint(v);
        w[2 * j + 1] = (uint32_t)__double2hiint(v);
    } else {
        w[j] = __float_as_uint(v);
    }
}

// Collision constants of a launch in the value type T (double, float, F2);
// rho0 is already multiplied by the run scale where the caller wants that.
template <class T> __device__ __forceinline__ Coef<T> coef_of(const RelaxBoth& r, double rho0);
template <> __device__ __forceinline__ Coef<double> coef_of<double>(const RelaxBoth& r, double rho0) {
    return make_coef<double>(r.d, rho0);
}
template <> __device__ __forceinline__ Coef<float> coef_of<float>(const RelaxBoth& r, double rho0) {
    return make_coef<float>(r.f, (float)rho0);
}
template <> __device__ __forceinline__ Coef<F2> coef_of<F2>(const RelaxBoth& r, double rho0) {
    return make_coef<F2>(r.f, (float)rho0);
}

// value type of the step kernel's collision: FP64 nodes one at a time;
// FP32-compute formats one node at a time (float) or two nodes at a time in
// packed FP32x2 (F2)
template <class S, bool PACKED> struct StepT { using T = typename std::conditional<PACKED, F2, float>::type; };
template <bool PACKED> struct StepT<double, PACKED> { using T = double; };

// The run scale, the scaled uniform force and G in the compute type C
// (precomputed on the host, derive_args).
template <class C> __device__ __forceinline__ C scale_of(const StepArgs& a) {
    if constexpr (sizeof(C) == 8) return a.scale; else return a.scale_f;
}
template <class C> __device__ __forceinline__ C fxs_of(const StepArgs& a) {
    if constexpr (sizeof(C) == 8) return a.fxs_d; else return a.fxs_f;
}
template <class C> __device__ __forceinline__ C fys_of(const StepArgs& a) {
    if constexpr (sizeof(C) == 8) return a.fys_d; else return a.fys_f;
}
template <class C> __device__ __forceinline__ C sc_g_of(const StepArgs& a) {
    if constexpr (sizeof(C) == 8) return a.sc_g; else return a.sc_g_f;
}

// Force at node (x, y) for the four force layouts of clbm_force_kind.
template <class C>
__device__ __forceinline__ void force_at(const StepArgs& a, int x, int y, C& Fx, C& Fy) {
    const C* F = static_cast<const C*>(a.force);
    switch (a.force_kind) {
        case 1: Fx = F[2 * y]; Fy = F[2 * y + 1]; break;
        case 2: Fx = F[2 * x]; Fy = F[2 * x + 1]; break;
        case 3: {
            const long long k = 2 * ((long long)y * a.geo.nx + x);
            Fx = F[k]; Fy = F[k + 1];
            break;
        }
        case 4:
            sc_force_node<C>(static_cast<const C*>(a.psi), a.geo.pitch, a.geo.nx, a.geo.ny, x, y,
                             (C)a.sc_g, Fx, Fy);
            break;
        default: Fx = (C)a.fx; Fy = (C)a.fy; break;
    }
}

// Two-node packed conversions for the 16-bit formats (one 32-bit word holds
// nodes j and j+1).
template <class S> struct Pair;
template <> struct Pair<__half> {
    __device__ static void decode(uint32_t w, float& lo, float& hi) {
        __half2 h;
        memcpy(&h, &w, 4);
        const float2 f = __half22float2(h);
        lo = f.x;
        hi = f.y;
    }
    __device__ static uint32_t encode(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ static void decode(uint32_t w, float& lo, float& hi) {
        lo = __uint_as_float(w << 16);
        hi = __uint_as_float(w & 0xffff0000u);
    }
    __device__ static uint32_t encode(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

// Stochastic rounding of the stores (clbm_set_rounding), by the sm_100-
// family conversion cvt.rs: each value rounds up when 16 random bits added
// below its kept mantissa carry into it, i.e. with probability equal to the
// dropped fraction (the upper 16 bits of the random word serve the upper
// value of the pair, the lower 16 the lower one; unbiased, as checked on
// the GPU over 2^20 draws).  The random words come from a counter-based
// hash: per node pair (2m, 2m + 1) of a row -- the pairs every launch shape
// stores together -- the 32-bit finaliser of MurmurHash3 (A. Appleby,
// public domain) of (first node, step); per population i of the pair, that
// hash times an odd constant of i, its upper half folded into the lower one
// (so the low bits of both halves, which the conversion takes, depend on the
// hash's low 29 bits, not on its low 13 alone).  A run is reproducible and
// every launch shape draws the same bits for a value.
__device__ __forceinline__ uint32_t sr_mix(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t sr_word(uint32_t pair_hash, uint32_t k) {
    const uint32_t r = pair_hash * ((2u * k + 1u) * 0x9e3779b9u);
    return r ^ (r >> 16);
}

template <> struct Pair<HalfSR> : Pair<__half> {
    __device__ static uint32_t encode_sr(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};
template <> struct Pair<Bf16SR> : Pair<__nv_bfloat16> {
    __device__ static uint32_t encode_sr(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};

// L2 prefetch of a contiguous byte range (16-byte aligned, multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, issued per thread; the
// data a thread copies is the data it later reads, so a thread's own
// cp.async.wait_group is the only synchronisation needed).
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? BYTES : 0;   // 0: zero-fill, nothing read
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES), "r"(n)
                     : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory stage of one warp (32-bit words):
//   planes [9][32 lanes][NW]      the 9 source vectors of each lane
//   edges  [6][32 lanes][EW]      left (planes 1, 5, 8) and right (3, 6, 7)
//                                 neighbour elements of the warp's edge lanes
//                                 (EW = 2 words for FP64, else 1)
//   mask   [32 lanes][2], solid [32 lanes]   (lattices with solid nodes)
//   own    [K][32 lanes][NW]      (lattices with solid nodes) the node's own
//                                 vectors of planes 4, 2, 7, 8, 5, 6 -- the
//                                 opposites that halfway bounce-back reads
//                                 for links 2, 4, 5, 6, 7, 8 (links 1, 3
//                                 read planes 3, 1, already in the stage)
// Row-chunk tasks give every lane K = 6 own slots, one per link.  Sparse
// and batch tasks (COMPACT) give each lane K = 2: the own vectors of links
// whose source row is all solid under the vector go into that row's plane
// slots (see own_cover), and a lane takes the rest in link order; the few
// lanes with more than two (obstacle corners, thickets of small obstacles)
// read the extra ones from global memory when they collide.  Along the
// sides of an obstacle a lane needs at most two, and the smaller stage lets
// four blocks of FP32 warps hold their rings on an SM instead of three
// (with the batch kernel's lattice descriptors in shared memory, see
// batch_step_kernel_staged).
//   pos    [32 lanes]             (sparse tasks) the lane's list entry,
//                                 written by the lane when it issues the
//                                 copies, so the collision does not read
//                                 the list again
template <int NW, bool MASK, int EW, int POS> struct Stage {
    static constexpr int kEW = EW;
    static constexpr int kOwnSlots = POS != 0 ? 2 : 6;
    static constexpr int kPlanes = 0;
    static constexpr int kEdges = 9 * 32 * NW;
    static constexpr int kMask = kEdges + 6 * 32 * EW;
    static constexpr int kSolid = kMask + 32 * 2;
    static constexpr int kOwn = kSolid + 32;
    static constexpr int kPos = MASK ? kOwn + kOwnSlots * 32 * NW : kMask;
    static constexpr int kWords = kPos + (POS == 2 ? 32 : 0);
    static_assert(kOwn % 4 == 0 && kWords % 4 == 0, "16-byte aligned vector slots");
};
template <class S, int NW, bool MASK, int POS = 0>
using StageOf = Stage<NW, MASK, sizeof(S) == 8 ? 2 : 1, POS>;

// The own vectors a lane reads for bounce-back: bit own_slot(i) for each
// link i in {2, 4, 5, 6, 7, 8} set at some fluid node of the vector (mw: link
// bytes, fluid: bit 8j set for a fluid node j).  The compact stage's own
// slots follow the bit order.
__device__ __forceinline__ uint32_t own_need(unsigned long long mw, unsigned long long fluid) {
    uint32_t need = 0u;
#pragma unroll
    for (int i = 2; i < 9; ++i) {
        if (i == 3) continue;
        if ((mw >> (i - 1)) & fluid) need |= 1u << own_slot(i);
    }
    return need;
}

// The own vectors that the compact stage puts into plane slots: where the
// source row of plane i under the vector is all solid, that row is not read,
// and every value taken from the slot (by this lane or, through the shuffle,
// by a neighbour) feeds a link that bounces; so the slot can hold the own
// vector of plane opp(i) that the bounce-back reads.  Along a flat wall this
// covers every bounce-back read.
__device__ __forceinline__ uint32_t own_cover(const bool row_solid[3]) {
    uint32_t cover = 0u;
#pragma unroll
    for (int i = 2; i < 9; ++i) {
        if (i == 3) continue;
        if (row_solid[ey_of(i) + 1]) cover |= 1u << own_slot(i);
    }
    return cover;
}

// Link word (byte j: link bits of node x0 + j) and solid flags of a chunk,
// read ahead of the chunk's copies so they can skip solid rows and fetch the
// bounce-back vectors.
constexpr uint32_t kSparseEnd = 0xffffffffu;

struct ChunkMask {
    unsigned long long mw = 0ull;
    uint32_t sflag = 0u;
    uint32_t e = kSparseEnd;   // sparse tasks: the lane's list entry
    uint32_t info = 0u;        // sparse tasks with masks: the entry's info word
};

// Where a lane works in a task: its row y, first node x0, whether it has
// nodes, and whether it fetches its left (right) neighbour element itself
// instead of taking it from lane - 1 (lane + 1).  POS selects the task form:
//   0  regular chunk (yt, c): 32 V consecutive nodes of row yt;
//   1  flat (batched steps): the task covers 32 consecutive vectors of the
//      lattice in row-major vector order, from vector c of row yt on (rows
//      of `chunks` vectors); it may run on into the next rows;
//   2  sparse: task yt holds entries 32 yt .. 32 yt + 31 of the lattice's
//      list of vectors with a fluid node (row << 16 | vector, row-major;
//      kSparseEnd past its end), one per lane.
struct LanePos {
    int y, x0;
    bool active, left, right;
};

// Sparse task position from the lane's list entry e (neighbour entries
// through the warp).
template <int V>
__device__ __forceinline__ LanePos lane_pos_entry(const StepArgs& a, uint32_t e, int lane) {
    LanePos p;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, e, 1);
    const uint32_t next = __shfl_down_sync(0xffffffffu, e, 1);
    p.active = e != kSparseEnd;
    p.y = p.active ? (int)(e >> 16) : 0;
    p.x0 = p.active ? (int)(e & 0xffffu) * V : 0;
    p.left = lane == 0 || prev == kSparseEnd || prev + 1u != e;
    p.right = lane == 31 || next == kSparseEnd || e + 1u != next || p.x0 + V >= a.geo.nx;
    return p;
}

template <int V, int POS>
__device__ __forceinline__ LanePos lane_pos(const StepArgs& a, int yt, int c, int lane) {
    LanePos p;
    if constexpr (POS == 2) return lane_pos_entry<V>(a, a.vlist[(long long)yt * 32 + lane], lane);
    if constexpr (POS == 1) {
        const int nvec = a.chunks;
        int xv = c + lane, y = yt;
        while (xv >= nvec) {
            xv -= nvec;
            ++y;
        }
        p.active = y < a.geo.ny;
        p.y = p.active ? y : yt;
        p.x0 = p.active ? xv * V : 0;
        p.left = lane == 0 || xv == 0;
    } else {
        p.y = yt;
        p.x0 = c * (32 * V) + lane * V;
        p.active = p.x0 < a.geo.nx;
        p.left = lane == 0;
    }
    p.right = lane == 31 || p.x0 + V >= a.geo.nx;
    return p;
}

template <class S, int NW>
__device__ __forceinline__ ChunkMask chunk_mask_at(const StepArgs& a, const LanePos& p) {
    constexpr int V = NW * 4 / (int)sizeof(S);
    ChunkMask m;
    const int x0 = p.x0, y = p.y;
    if (!p.active) {
        m.mw = V == 8 ? ~0ull : ((1ull << (8 * V)) - 1ull);
        m.sflag = (1u << V) - 1u;
        return m;
    }
    const long long q = (long long)y * a.geo.pitch + x0;
    const uint8_t* mp = a.lmask + q;
    if constexpr (V == 2) {
        m.mw = *reinterpret_cast<const unsigned short*>(mp);
    } else if constexpr (V == 4) {
        m.mw = *reinterpret_cast<const unsigned int*>(mp);
    } else {
        m.mw = *reinterpret_cast<const unsigned long long*>(mp);
    }
    m.sflag = ((uint32_t)a.sbits[q >> 3] >> (q & 7)) & ((1u << V) - 1u);
    return m;
}

template <class S, int NW, int POS = 0>
__device__ __forceinline__ ChunkMask load_chunk_mask(const StepArgs& a, int yt, int c, int lane) {
    constexpr int V = NW * 4 / (int)sizeof(S);
    return chunk_mask_at<S, NW>(a, lane_pos<V, POS>(a, yt, c, lane));
}

// A sparse task's ChunkMask: the lane's list entry and, with masks, its info
// word (both read ahead); the link bits go to the stage with the copies.
__device__ __forceinline__ ChunkMask sparse_entry(uint32_t e, uint32_t info) {
    ChunkMask m;
    m.e = e;
    m.info = info;
    return m;
}

// L1 prefetch of the line holding p (the force values a chunk will read).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// This step's hash seed of stochastic rounding (the device step counter
// does not change during a launch).
template <class S>
__device__ __forceinline__ uint32_t sr_seed_of(const StepArgs& a) {
    if constexpr (Stochastic<S>::value) return sr_mix(__ldg(a.sr_step) * 0x9e3779b9u);
    else return 0u;
}

__host__ __device__ constexpr int edge_slot(int i) {
    return i == 1 ? 0 : i == 5 ? 1 : i == 8 ? 2 : i == 3 ? 3 : i == 6 ? 4 : 5;
}

// Copy the element at p (FP64/FP32), or the aligned 32-bit word holding it
// (16-bit formats), into an edge slot.
template <class S>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const S* p, bool valid) {
    if constexpr (sizeof(S) == 8) {
        cp_async<8>(dst, p, valid);
    } else if constexpr (sizeof(S) == 4) {
        cp_async<4>(dst, p, valid);
    } else {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(3);
        cp_async<4>(dst, reinterpret_cast<const void*>(a), valid);
    }
}

// The element of edge slot e of this lane; xi is the element's column (its
// parity selects the half of a 16-bit word).
template <class S>
__device__ __forceinline__ typename Raw<S>::E stage_elem(const uint32_t* stg, int e, int lane, int xi) {
    // stg points at the edge slots: EW = 2 words per slot for FP64, else 1
    const uint32_t* q = stg + (e * 32 + lane) * (sizeof(S) == 8 ? 2 : 1);
    if constexpr (sizeof(S) == 8) {
        return ((unsigned long long)q[1] << 32) | q[0];
    } else if constexpr (sizeof(S) == 4) {
        return q[0];
    } else {
        return (xi & 1) ? (q[0] >> 16) : (q[0] & 0xffffu);
    }
}

// Issue the copies of chunk (yt, c) into this lane's slots of stage stg.
template <class S, int NW, bool MASK, int POS = 0>
__device__ __forceinline__ void issue_chunk(const StepArgs& a, const void* srcp, int yt, int c, int lane,
                                            uint32_t* stg, const ChunkMask& cm) {
    // (sparse tasks: cm carries the lane's list entry; yt, c are unused)
    using St = StageOf<S, NW, MASK, POS>;
    constexpr int V = NW * 4 / (int)sizeof(S);
    const int nx = a.geo.nx, ny = a.geo.ny, pitch = a.geo.pitch;
    const long long plane = a.geo.plane;
    LanePos p;
    if constexpr (POS == 2) {
        p = lane_pos_entry<V>(a, cm.e, lane);   // the entry was read with the mask
        stg[St::kPos + lane] = cm.e;
    } else {
        p = lane_pos<V, POS>(a, yt, c, lane);
    }
    const int x0 = p.x0, y = p.y;
    const bool active = p.active;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const S* src = static_cast<const S*>(srcp);
    const S* rowb[3] = {src + (long long)yp * pitch, src + (long long)y * pitch,
                        src + (long long)ym * pitch};
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(stg);
    const int xs = active ? x0 : 0;
    // the force values the collision will read, into L1 ahead of it
    if (active && a.force_kind >= 1 && a.force_kind <= 3) {
        using C = typename Fmt<S>::C;
        const C* Fa = static_cast<const C*>(a.force);
        prefetch_l1(Fa + (a.force_kind == 1   ? 2LL * y
                          : a.force_kind == 2 ? 2LL * x0
                                              : 2LL * ((long long)y * nx + x0)));
    }
    // rows whose positions under this vector are all solid are not read
    // (their values would all be replaced by bounce-back)
    bool row_solid[3] = {false, false, false};
    unsigned long long fluid = 0ull;          // bit 8j: node x0 + j is fluid
    bool plain = true;
    if constexpr (MASK && POS == 2) {         // sparse: from the info word
        plain = !(cm.info & kInfoNotPlain);
#pragma unroll
        for (int r = 0; r < 3; ++r) row_solid[r] = (cm.info >> (kInfoRowShift + r)) & 1u;
    } else if constexpr (MASK) {
        plain = cm.mw == 0ull && cm.sflag == 0u;
        if (!plain) {
            uint32_t all = 0xff;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                all &= (uint32_t)(cm.mw >> (8 * j)) & 0xffu;
                if (!((cm.sflag >> j) & 1u)) fluid |= 1ull << (8 * j);
            }
            row_solid[0] = (all >> 3) & 1u;
            row_solid[1] = cm.sflag == (1u << V) - 1u;
            row_solid[2] = (all >> 1) & 1u;
        }
    }
    // own vectors of the opposite planes, for the links that bounce (the
    // compact layout puts some of them into plane slots)
    uint32_t need = 0u, cover = 0u;
    if constexpr (MASK && POS == 2) {         // cover: only the slots that are read
        cover = (cm.info >> kInfoCoverShift) & 0x3fu;
        need = cover | ((cm.info >> kInfoRestShift) & 0x3fu);
    } else if constexpr (MASK) {
        if (active && !plain) {
            need = own_need(cm.mw, fluid);
            if constexpr (St::kOwnSlots == 2) cover = own_cover(row_solid);
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int r = ey_of(i) + 1;
        const uint32_t dst = sb + 4u * (St::kPlanes + (i * 32 + lane) * NW);
        if (St::kOwnSlots == 2 && MASK && r != 1 && row_solid[r]) {   // own vector opp(i)
            cp_async<NW * 4>(dst, rowb[1] + opp_of(i) * plane + xs, (cover & need) >> own_slot(i) & 1u);
        } else {
            cp_async<NW * 4>(dst, rowb[r] + i * plane + xs, active && !row_solid[r]);
        }
    }
    if constexpr (MASK) {
        need &= ~cover;
        if (need) {
#pragma unroll
            for (int i = 2; i < 9; ++i) {
                if (i == 3) continue;
                const uint32_t bit = 1u << own_slot(i);
                if constexpr (St::kOwnSlots == 6) {
                    if (need & bit)
                        cp_async<NW * 4>(sb + 4u * (St::kOwn + (own_slot(i) * 32 + lane) * NW),
                                         rowb[1] + opp_of(i) * plane + x0, true);
                } else {
                    const int k = __popc(need & (bit - 1u));    // rank among the lane's reads
                    if ((need & bit) && k < 2)
                        cp_async<NW * 4>(sb + 4u * (St::kOwn + (k * 32 + lane) * NW),
                                         rowb[1] + opp_of(i) * plane + x0, true);
                }
            }
        }
    }
    // edge elements: node 0 takes the left one, the last node of the row in
    // the vector the right one.  Sparse tasks (many run ends, mostly beside
    // solid nodes) skip them where that node is solid or the link bounces
    // (info bits kInfoLeftShift + edge slot: left slots 0-2, right 3-5).
    constexpr bool kSkipEdges = MASK && POS == 2;
    if (p.left && active) {
        const int xl = x0 == 0 ? nx - 1 : x0 - 1;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (ex_of(i) <= 0) continue;
            const bool use = !kSkipEdges || plain || ((cm.info >> (kInfoLeftShift + edge_slot(i))) & 1u);
            cp_async_elem<S>(sb + 4u * (St::kEdges + (edge_slot(i) * 32 + lane) * St::kEW),
                             rowb[ey_of(i) + 1] + i * plane + xl, use);
        }
    }
    if (p.right && active) {
        const int xr = x0 + V >= nx ? 0 : x0 + V;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (ex_of(i) >= 0) continue;
            const bool use = !kSkipEdges || plain || ((cm.info >> (kInfoLeftShift + edge_slot(i))) & 1u);
            cp_async_elem<S>(sb + 4u * (St::kEdges + (edge_slot(i) * 32 + lane) * St::kEW),
                             rowb[ey_of(i) + 1] + i * plane + xr, use);
        }
    }
    if constexpr (MASK) {
        const long long q = (long long)y * pitch + xs;
        const uint32_t dm = sb + 4u * (St::kMask + lane * 2);
        if constexpr (V == 2) {
            cp_async<4>(dm, a.lmask + (q & ~3LL), active);
        } else if constexpr (V == 4) {
            cp_async<4>(dm, a.lmask + q, active);
        } else {
            cp_async<8>(dm, a.lmask + q, active);
        }
        if constexpr (POS == 2)   // sparse: the info word (solid flags included)
            stg[St::kSolid + lane] = cm.info;
        else
            cp_async<4>(sb + 4u * (St::kSolid + lane), a.sbits + ((q >> 3) & ~3LL), active);
    }
}

// ---------------------------------------------------------------------------
// The fused step kernel.  A persistent grid of warps walks the row chunks
// (one chunk = 32 * V consecutive nodes of one row, V = 4 * NW / element
// size); before working on a chunk a warp asks L2 for the source rows of its
// next chunk, so DRAM keeps streaming while the warp computes.
// MASK = the lattice has solid nodes.
// All arithmetic runs on deviations scaled by 2^k: rho0 and F are scaled
// once, u = j / rho is scale-free, and the collision is otherwise linear.
// ---------------------------------------------------------------------------
// One chunk of one lattice: `a` describes the lattice (it may live in
// global memory for batched launches), srcp/dstp are its current source and
// destination population planes.
template <class S, int NW, bool MASK, bool PACKED, bool STAGED, bool GUO = false, int POS = 0,
          bool SC = false>
__device__ __forceinline__ void step_chunk(const StepArgs& a, const void* srcp, void* dstp, int yt,
                                           int c, int lane,
                                           const Coef<typename StepT<S, PACKED>::T>& kc,
                                           const uint32_t* stg, uint32_t sr_seed = 0u) {
    using C = typename Fmt<S>::C;
    using E = typename Raw<S>::E;
    constexpr int V = NW * 4 / (int)sizeof(S);
    constexpr bool PAIRED = is16<S>::value;

    const int nx = a.geo.nx, ny = a.geo.ny, pitch = a.geo.pitch;
    const long long plane = a.geo.plane;
    LanePos lp;
    if constexpr (POS == 2 && STAGED)   // sparse: the entry the lane staged at issue
        lp = lane_pos_entry<V>(a, stg[StageOf<S, NW, MASK, POS>::kPos + lane], lane);
    else
        lp = lane_pos<V, POS>(a, yt, c, lane);
    const int x0 = lp.x0, y = lp.y;
    const bool active = lp.active;
    const int ym = (y == 0) ? ny - 1 : y - 1;      // source row of e_y = +1
    const int yp = (y == ny - 1) ? 0 : y + 1;      // source row of e_y = -1
    const S* src = static_cast<const S*>(srcp);
    const S* rowb[3] = {src + (long long)yp * pitch, src + (long long)y * pitch,
                        src + (long long)ym * pitch};   // indexed by e_y + 1

    // link bits of the V nodes (bit i-1 set: the source x - e_i is solid)
    // and their solid flags (bitmap, one bit per node)
    // Byte j of mw holds the link bits of node x0 + j; sflag bit j its solid
    // flag.  `plain` vectors (no link bit, no solid node -- almost all of a
    // lattice) skip every bounce-back and solid-node step below.
    unsigned long long mw = 0ull;
    uint32_t sflag = 0u;
    uint32_t info = 0u;     // sparse staged tasks: the entry's info word
    constexpr bool kInfo = MASK && STAGED && POS == 2;
    bool all_solid = false, plain = true;
    bool row_solid[3] = {false, false, false};     // source rows e_y = -1, 0, +1 all solid
    if constexpr (MASK) {
        const long long q = (long long)y * pitch + x0;
        if (active && STAGED) {
            using St = StageOf<S, NW, MASK, POS>;
            const uint32_t m0 = stg[St::kMask + lane * 2], m1 = stg[St::kMask + lane * 2 + 1];
            if constexpr (V == 2) {
                mw = (m0 >> (8 * (q & 3))) & 0xffffu;
            } else if constexpr (V == 4) {
                mw = m0;
            } else {
                mw = ((unsigned long long)m1 << 32) | m0;
            }
            if constexpr (kInfo) {
                info = stg[St::kSolid + lane];
                sflag = info & ((1u << V) - 1u);
            } else {
                const uint32_t sw = stg[St::kSolid + lane];
                sflag = (sw >> (8 * ((q >> 3) & 3) + (q & 7))) & ((1u << V) - 1u);
            }
        } else if (active) {
            const uint8_t* mp = a.lmask + q;
            if constexpr (V == 2) {
                mw = *reinterpret_cast<const unsigned short*>(mp);
            } else if constexpr (V == 4) {
                mw = *reinterpret_cast<const unsigned int*>(mp);
            } else {
                mw = *reinterpret_cast<const unsigned long long*>(mp);
            }
            // pitch is a multiple of 8, so the V flags sit in one byte
            sflag = ((uint32_t)a.sbits[q >> 3] >> (q & 7)) & ((1u << V) - 1u);
        } else {
            mw = V == 8 ? ~0ull : ((1ull << (8 * V)) - 1ull);
            sflag = (1u << V) - 1u;
        }
        if constexpr (kInfo) {
            plain = !active || !(info & kInfoNotPlain);
            all_solid = sflag == (1u << V) - 1u;
#pragma unroll
            for (int r = 0; r < 3; ++r) row_solid[r] = (info >> (kInfoRowShift + r)) & 1u;
        } else {
            plain = (mw == 0ull) && (sflag == 0u);
            if (!plain) {
                uint32_t all = 0xff;
#pragma unroll
                for (int j = 0; j < V; ++j) all &= (uint32_t)(mw >> (8 * j)) & 0xffu;
                all_solid = sflag == (1u << V) - 1u;
                // link 2 (source (x, y-1)) and link 4 (source (x, y+1)) give
                // the solidity of the neighbouring rows under this vector
                row_solid[0] = (all >> 3) & 1u;
                row_solid[1] = all_solid;
                row_solid[2] = (all >> 1) & 1u;
            }
        }
    }

    // ---- a1: pull-stream (Eq. 10) ------------------------------------------
    uint32_t w[9][NW];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ey = ey_of(i);
        const bool load = active && !row_solid[ey + 1];
        if constexpr (STAGED) {
            const uint32_t* q = stg + StageOf<S, NW, MASK, POS>::kPlanes + (i * 32 + lane) * NW;
            if constexpr (NW == 4) {
                const uint4 v = *reinterpret_cast<const uint4*>(q);
                w[i][0] = v.x; w[i][1] = v.y; w[i][2] = v.z; w[i][3] = v.w;
            } else {
                const uint2 v = *reinterpret_cast<const uint2*>(q);
                w[i][0] = v.x; w[i][1] = v.y;
            }
        } else if (load) {
            ld_vec<NW>(rowb[ey + 1] + i * plane + x0, w[i]);
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k) w[i][k] = 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ex = ex_of(i), ey = ey_of(i);
        if (ex == 0) continue;
        const S* rowp = rowb[ey + 1] + i * plane;
        if (ex > 0) {           // source x - 1
            E L = __shfl_up_sync(0xffffffffu, raw_get<S, NW>(w[i], V - 1), 1);
            if (lp.left && active) {
                const int xl = x0 == 0 ? nx - 1 : x0 - 1;
                if constexpr (STAGED) {
                    L = stage_elem<S>(stg + StageOf<S, NW, MASK, POS>::kEdges, edge_slot(i), lane, xl);
                } else {
                    L = ld_elem<S>(rowp + xl);
                }
            }
            shift_in_left<S, NW>(w[i], L);
        } else {                // source x + 1
            E R = __shfl_down_sync(0xffffffffu, raw_get<S, NW>(w[i], 0), 1);
            const bool edge = lp.right;
            if (edge && active) {
                const int xr = x0 + V >= nx ? 0 : x0 + V;
                if constexpr (STAGED) {
                    R = stage_elem<S>(stg + StageOf<S, NW, MASK, POS>::kEdges, edge_slot(i), lane, xr);
                } else {
                    R = ld_elem<S>(rowp + xr);
                }
            }
            shift_in_right<S, NW>(w[i], R);
            if (active && x0 + V > nx) {   // ragged row end: node nx-1 wraps to x = 0
                const int jr = nx - 1 - x0;
#pragma unroll
                for (int j = 0; j < V - 1; ++j)
                    if (j == jr) raw_set<S, NW>(w[i], j, R);
            }
        }
    }

    // ---- a1: halfway bounce-back (Sec. 4A): f_i(x) = f*_opp(i)(x) ---------
    if constexpr (MASK) {
        if (active && !plain && !all_solid) {
            // one bit per byte: fluid nodes of the vector
            unsigned long long fluid = 0ull;
            // compact stage: own vectors in plane slots (cover), the rest in
            // the lane's two own slots in link order, or read here
            uint32_t rest = 0u, cover = 0u;
            if constexpr (kInfo) {      // the plan computed on the host
                cover = (info >> kInfoCoverShift) & 0x3fu;
                rest = (info >> kInfoRestShift) & 0x3fu;
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (!((sflag >> j) & 1u)) fluid |= 1ull << (8 * j);
                if constexpr (STAGED && StageOf<S, NW, MASK, POS>::kOwnSlots == 2) {
                    cover = own_cover(row_solid);
                    rest = own_need(mw, fluid) & ~cover;
                }
            }
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const bool bounces =
                    kInfo ? (i == 1   ? (info >> kInfoBounce1) & 1u
                             : i == 3 ? (info >> kInfoBounce3) & 1u
                                      : ((cover | rest) >> own_slot(i)) & 1u) != 0u
                          : ((mw >> (i - 1)) & fluid) != 0ull;
                if (bounces) {
                    uint32_t o[NW];
                    if constexpr (STAGED) {
                        using St = StageOf<S, NW, MASK, POS>;
                        const bool row = i == 1 || i == 3;
                        if constexpr (St::kOwnSlots == 6) {
                            const uint32_t* q = row ? stg + St::kPlanes + (opp_of(i) * 32 + lane) * NW
                                                    : stg + St::kOwn + (own_slot(i) * 32 + lane) * NW;
#pragma unroll
                            for (int k = 0; k < NW; ++k) o[k] = q[k];
                        } else {
                            const bool cov = !row && ((cover >> own_slot(i)) & 1u);
                            const int k = __popc(rest & ((1u << own_slot(i)) - 1u));
                            if (row || cov || k < 2) {
                                const uint32_t* q = row ? stg + St::kPlanes + (opp_of(i) * 32 + lane) * NW
                                                    : cov ? stg + St::kPlanes + (i * 32 + lane) * NW
                                                          : stg + St::kOwn + (k * 32 + lane) * NW;
#pragma unroll
                                for (int m = 0; m < NW; ++m) o[m] = q[m];
                            } else {
                                ld_vec<NW>(rowb[1] + opp_of(i) * plane + x0, o);
                            }
                        }
                    } else {
                        ld_vec<NW>(rowb[1] + opp_of(i) * plane + x0, o);
                    }
                    link_select<S, NW>(w[i], o, mw >> (i - 1));
                }
            }
        }
    }

    // ---- body force of the V nodes (kind is uniform over the launch) -------
    C Fx[V], Fy[V];
    if constexpr (SC) {       // Shan-Chen (Sec. 4C), from this step's psi field
        const C sc = scale_of<C>(a);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            C fx, fy;
            sc_force_node<C>(static_cast<const C*>(a.psi), pitch, nx, ny, min(x0 + j, nx - 1), y,
                             sc_g_of<C>(a), fx, fy);
            Fx[j] = Alg<C>::mul(fx, sc);
            Fy[j] = Alg<C>::mul(fy, sc);
        }
    } else {
        const C* Fa = static_cast<const C*>(a.force);
        const C sc = scale_of<C>(a);
        if (a.force_kind == 1) {
            const C fx = Fa[2 * y] * sc, fy = Fa[2 * y + 1] * sc;
#pragma unroll
            for (int j = 0; j < V; ++j) { Fx[j] = fx; Fy[j] = fy; }
        } else if (a.force_kind == 2 || a.force_kind == 3) {
            const long long base = a.force_kind == 2 ? 0 : (long long)y * nx;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const long long k = 2 * (base + min(x0 + j, nx - 1));
                Fx[j] = Fa[k] * sc;
                Fy[j] = Fa[k + 1] * sc;
            }
        } else {
            const C fx = fxs_of<C>(a), fy = fys_of<C>(a);
#pragma unroll
            for (int j = 0; j < V; ++j) { Fx[j] = fx; Fy[j] = fy; }
        }
    }

    // ---- a2-a7: collide every node of the vector, encode in place ---------
    // (stochastic rounding: per node pair, a hash of the node and this
    // step's seed, sr_seed_of)
    uint32_t sr_pair[V / 2];
    if constexpr (Stochastic<S>::value) {
#pragma unroll
        for (int p = 0; p < V / 2; ++p) sr_pair[p] = sr_mix((uint32_t)(y * pitch + x0 + 2 * p) ^ sr_seed);
    }
    // (a8: a fully solid vector is neither computed nor stored)
    if (MASK && all_solid) return;
    if constexpr (sizeof(S) == 8) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            double g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = elem_get<S, NW>(w[i], j);
            collide<double, GUO>(g, Fx[j], Fy[j], kc);
            if (MASK && ((sflag >> j) & 1u)) {
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = 0.0;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) elem_set<S, NW>(w[i], j, g[i]);
        }
    } else if constexpr (!PACKED) {
#pragma unroll
        for (int p = 0; p < V / 2; ++p) {       // nodes 2p and 2p+1, one at a time
            float g0[9], g1[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if constexpr (PAIRED) {
                    Pair<S>::decode(w[i][p], g0[i], g1[i]);
                } else {
                    g0[i] = __uint_as_float(w[i][2 * p]);
                    g1[i] = __uint_as_float(w[i][2 * p + 1]);
                }
            }
            collide<float, GUO>(g0, Fx[2 * p], Fy[2 * p], kc);
            collide<float, GUO>(g1, Fx[2 * p + 1], Fy[2 * p + 1], kc);
            if (MASK && ((sflag >> (2 * p)) & 3u)) {
                const bool s0 = (sflag >> (2 * p)) & 1u, s1 = (sflag >> (2 * p + 1)) & 1u;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    g0[i] = s0 ? 0.0f : g0[i];
                    g1[i] = s1 ? 0.0f : g1[i];
                }
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float lo = g0[i];
                const float hi = g1[i];
                if constexpr (Stochastic<S>::value) {
                    w[i][p] = Pair<S>::encode_sr(lo, hi, sr_word(sr_pair[p], (uint32_t)i));
                } else if constexpr (PAIRED) {
                    w[i][p] = Pair<S>::encode(lo, hi);
                } else {
                    w[i][2 * p] = __float_as_uint(lo);
                    w[i][2 * p + 1] = __float_as_uint(hi);
                }
            }
        }
    } else {
#pragma unroll
        for (int p = 0; p < V / 2; ++p) {       // nodes 2p and 2p+1 as one F2
            F2 g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float lo, hi;
                if constexpr (PAIRED) {
                    Pair<S>::decode(w[i][p], lo, hi);
                } else {
                    lo = __uint_as_float(w[i][2 * p]);
                    hi = __uint_as_float(w[i][2 * p + 1]);
                }
                g[i].v = make_float2(lo, hi);
            }
            collide<F2, GUO>(g, F2{make_float2(Fx[2 * p], Fx[2 * p + 1])},
                        F2{make_float2(Fy[2 * p], Fy[2 * p + 1])}, kc);
            if (MASK && ((sflag >> (2 * p)) & 3u)) {
                const bool s0 = (sflag >> (2 * p)) & 1u, s1 = (sflag >> (2 * p + 1)) & 1u;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    g[i].v.x = s0 ? 0.0f : g[i].v.x;
                    g[i].v.y = s1 ? 0.0f : g[i].v.y;
                }
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float lo = g[i].v.x;
                const float hi = g[i].v.y;
                if constexpr (Stochastic<S>::value) {
                    w[i][p] = Pair<S>::encode_sr(lo, hi, sr_word(sr_pair[p], (uint32_t)i));
                } else if constexpr (PAIRED) {
                    w[i][p] = Pair<S>::encode(lo, hi);
                } else {
                    w[i][2 * p] = __float_as_uint(lo);
                    w[i][2 * p + 1] = __float_as_uint(hi);
                }
            }
        }
    }

    // ---- a7: store (a8: fully solid vectors write nothing) -----------------
    if (active && !all_solid) {
        S* dst = static_cast<S*>(dstp) + (long long)y * pitch + x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_vec<NW>(dst + i * plane, w[i]);
    }
}

// lanes 0..8 ask L2 for plane `lane` of chunk (y, c): its source row segment
template <class S, int NW>
__device__ __forceinline__ void prefetch_chunk(const StepArgs& a, int y, int c, int lane) {
    constexpr int V = NW * 4 / (int)sizeof(S);
    if (lane >= 9) return;
    const int ey = ey_of(lane);
    const int row = ey > 0 ? (y == 0 ? a.geo.ny - 1 : y - 1)
                           : (ey < 0 ? (y == a.geo.ny - 1 ? 0 : y + 1) : y);
    const int x0 = c * 32 * V;
    const int n = min(32 * V, a.geo.pitch - x0);
    const S* p = static_cast<const S*>(a.src) + lane * a.geo.plane + (long long)row * a.geo.pitch + x0;  // single lattice
    prefetch_l2(p, (uint32_t)(n * (int)sizeof(S)));
}

constexpr int kStepThreads = 128;

template <class S, int NW, bool MASK, bool PACKED, bool GUO, bool SC>
__global__ void __launch_bounds__(kStepThreads) step_kernel(const StepArgs a) {
    using T = typename StepT<S, PACKED>::T;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const Coef<T> kc = coef_of<T>(a.relax, a.rho0 * a.scale);
    const uint32_t seed = sr_seed_of<S>(a);
    // walk the tasks (row, chunk) with a stride of nwarps, in 32-bit steps
    const int chunks = a.chunks;
    const int t0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y = t0 / chunks, c = t0 - (t0 / chunks) * chunks;
    const int dy = nwarps / chunks, dc = nwarps - dy * chunks;
    // prefetch cursor: `dist` strides ahead of (y, c)
    const int dist = a.prefetch;
    int py = y, pc = c;
    for (int k = 0; k < dist; ++k) {
        py += dy;
        pc += dc;
        if (pc >= chunks) { pc -= chunks; ++py; }
        if (k + 1 < dist && py < a.geo.ny) prefetch_chunk<S, NW>(a, py, pc, lane);
    }
    while (y < a.geo.ny) {
        if (dist > 0) {
            if (py < a.geo.ny) prefetch_chunk<S, NW>(a, py, pc, lane);
            py += dy;
            pc += dc;
            if (pc >= chunks) { pc -= chunks; ++py; }
        }
        step_chunk<S, NW, MASK, PACKED, false, GUO, 0, SC>(a, a.src, a.dst, y, c, lane, kc, nullptr, seed);
        y += dy;
        c += dc;
        if (c >= chunks) { c -= chunks; ++y; }
    }
}

// Threads per block of the staged row-chunk kernel: one warp for the
// 16-bit formats, four otherwise.  The FP16 and BF16 kernels hold 134
// registers a thread, so four-warp blocks fit three to an SM (12 warps)
// where one-warp blocks fit 15.  Measured at 8192^2 against four-warp
// blocks: FP16 0.934 -> 0.940 and BF16 0.948 -> 0.952 of HBM, with
// stochastic rounding (128 registers, 16 warps either way) 0.789 -> 0.833
// and 0.813 -> 0.855; FP32 runs faster in four-warp blocks (0.915 against
// 0.897), as do the sparse-list kernels.
template <class S>
constexpr int staged_threads() {
    return is16<S>::value ? 32 : kStepThreads;
}

// The step kernel with a shared-memory ring of ST stages per warp: while a
// warp computes chunk k, the copies of its chunks k+1 .. k+ST-1 are in
// flight (cp.async), so DRAM latency is hidden without extra registers.
// GUO: the M2 forcing terms; SC: the Shan-Chen force from the psi field
// (both on lattices without solid nodes, in the default shape only).  RL:
// the rows are a.rowlist[0 .. a.nrows - 1] (a sparse lattice's rows of
// plain vectors) instead of 0 .. ny - 1.
template <class S, int NW, bool MASK, bool PACKED, int ST, bool GUO = false, bool SC = false, bool RL = false>
__global__ void __launch_bounds__(staged_threads<S>()) step_kernel_staged(const StepArgs a) {
    using T = typename StepT<S, PACKED>::T;
    constexpr int SW = StageOf<S, NW, MASK>::kWords;
    extern __shared__ __align__(16) uint32_t smem_stage[];
    const int lane = threadIdx.x & 31;
    uint32_t* wb = smem_stage + (threadIdx.x >> 5) * ST * SW;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const Coef<T> kc = coef_of<T>(a.relax, a.rho0 * a.scale);
    const uint32_t seed = sr_seed_of<S>(a);
    const int chunks = a.chunks, ny = RL ? a.nrows : a.geo.ny;   // rows to step
    auto row = [&](int r) -> int {            // row r of the ones to step
        if constexpr (RL) return __ldg(a.rowlist + r);
        else return r;
    };
    const int t0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int y = t0 / chunks, c = t0 - (t0 / chunks) * chunks;
    const int dy = nwarps / chunks, dc = nwarps - dy * chunks;
    int iy = y, ic = c;                         // issue cursor
#pragma unroll
    for (int st = 0; st < ST - 1; ++st) {
        if (iy < ny) {
            ChunkMask cm;
            if constexpr (MASK) cm = load_chunk_mask<S, NW>(a, row(iy), ic, lane);
            issue_chunk<S, NW, MASK>(a, a.src, row(iy), ic, lane, wb + st * SW, cm);
        }
        cp_async_commit();
        iy += dy;
        ic += dc;
        if (ic >= chunks) { ic -= chunks; ++iy; }
    }
    // masks are read one iteration before their chunk is issued
    ChunkMask nxt;
    if constexpr (MASK) {
        if (iy < ny) nxt = load_chunk_mask<S, NW>(a, row(iy), ic, lane);
    }
    int slot = 0;
    while (y < ny) {
        cp_async_wait<ST - 2>();                // this lane's copies of chunk (y, c) landed
        const int islot = slot == 0 ? ST - 1 : slot - 1;   // stage freed last iteration
        if (iy < ny) issue_chunk<S, NW, MASK>(a, a.src, row(iy), ic, lane, wb + islot * SW, nxt);
        cp_async_commit();
        iy += dy;
        ic += dc;
        if (ic >= chunks) { ic -= chunks; ++iy; }
        if constexpr (MASK) {
            if (iy < ny) nxt = load_chunk_mask<S, NW>(a, row(iy), ic, lane);
        }
        step_chunk<S, NW, MASK, PACKED, true, GUO, 0, SC>(a, a.src, a.dst, row(y), c, lane, kc, wb + slot * SW, seed);
        y += dy;
        c += dc;
        if (c >= chunks) { c -= chunks; ++y; }
        slot = slot + 1 == ST ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

// Sparse forms of the masked step for lattices whose solid nodes fill many
// whole vectors: the tasks are groups of 32 entries of the list of vectors
// holding a fluid node, so no lane is spent on an all-solid vector.  The
// list comes in two parts: plain vectors (no link bit, no solid node: the
// step there is that of a lattice without walls, MASK = false) and the
// rest (MASK = true); each part is one launch.  Same per-node arithmetic as
// the (row, chunk) kernels, hence the same bits.
template <class S, int NW, bool MASK, bool PACKED>
__global__ void __launch_bounds__(kStepThreads) step_kernel_sparse(const StepArgs a) {
    using T = typename StepT<S, PACKED>::T;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const Coef<T> kc = coef_of<T>(a.relax, a.rho0 * a.scale);
    const uint32_t seed = sr_seed_of<S>(a);
    for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < a.vtasks; t += nwarps)
        step_chunk<S, NW, MASK, PACKED, false, false, 2>(a, a.src, a.dst, t, 0, lane, kc, nullptr, seed);
}

template <class S, int NW, bool MASK, bool PACKED, int ST>
__device__ __forceinline__ void sparse_staged_body(const StepArgs& a) {
    using T = typename StepT<S, PACKED>::T;
    constexpr int SW = StageOf<S, NW, MASK, 2>::kWords;
    extern __shared__ __align__(16) uint32_t smem_stage[];
    const int lane = threadIdx.x & 31;
    uint32_t* wb = smem_stage + (threadIdx.x >> 5) * ST * SW;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const Coef<T> kc = coef_of<T>(a.relax, a.rho0 * a.scale);
    const uint32_t seed = sr_seed_of<S>(a);
    const int ntasks = a.vtasks;
    // list entry and info word of task k (kSparseEnd past the list)
    auto entry = [&](int k) {
        return k < ntasks ? __ldg(a.vlist + (long long)k * 32 + lane) : kSparseEnd;
    };
    auto info = [&](int k) {
        return MASK && k < ntasks ? __ldg(a.vinfo + (long long)k * 32 + lane) : 0u;
    };
    int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int ti = t;                                 // issue cursor
#pragma unroll
    for (int st = 0; st < ST - 1; ++st) {
        if (ti < ntasks) issue_chunk<S, NW, MASK, 2>(a, a.src, 0, 0, lane, wb + st * SW,
                                                     sparse_entry(entry(ti), info(ti)));
        cp_async_commit();
        ti += nwarps;
    }
    // the list entries and info words are read two issues ahead, so those
    // reads do not wait on memory where they are used
    ChunkMask nxt;
    if (ti < ntasks) nxt = sparse_entry(entry(ti), info(ti));
    uint32_t e_ahead = entry(ti + nwarps), i_ahead = info(ti + nwarps);
    int slot = 0;
    while (t < ntasks) {
        cp_async_wait<ST - 2>();
        const int islot = slot == 0 ? ST - 1 : slot - 1;
        if (ti < ntasks) issue_chunk<S, NW, MASK, 2>(a, a.src, 0, 0, lane, wb + islot * SW, nxt);
        cp_async_commit();
        ti += nwarps;
        if (ti < ntasks) nxt = sparse_entry(e_ahead, i_ahead);
        e_ahead = entry(ti + nwarps);
        i_ahead = info(ti + nwarps);
        step_chunk<S, NW, MASK, PACKED, true, false, 2>(a, a.src, a.dst, t, 0, lane, kc, wb + slot * SW, seed);
        t += nwarps;
        slot = slot + 1 == ST ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

template <class S, int NW, bool MASK, bool PACKED, int ST>
__global__ void __launch_bounds__(kStepThreads) step_kernel_sparse_staged(const StepArgs a) {
    sparse_staged_body<S, NW, MASK, PACKED, ST>(a);
}

template <class S, int NW, bool MASK, bool PACKED, int ST>
static cudaError_t sparse_launch(const StepArgs& a, cudaStream_t s) {
    constexpr int SW = StageOf<S, NW, MASK, 2>::kWords;
    constexpr int kSmem = ST > 0 ? (kStepThreads / 32) * ST * SW * 4 : 0;
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if constexpr (ST > 0) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(step_kernel_sparse_staged<S, NW, MASK, PACKED, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, step_kernel_sparse_staged<S, NW, MASK, PACKED, ST>, kStepThreads, kSmem);
        } else {
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, step_kernel_sparse<S, NW, MASK, PACKED>, kStepThreads, 0);
        }
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int wpb = kStepThreads / 32;
    const int need = (a.vtasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    if (blocks == 0) return cudaSuccess;
    if constexpr (ST > 0)
        step_kernel_sparse_staged<S, NW, MASK, PACKED, ST><<<blocks, kStepThreads, kSmem, s>>>(a);
    else
        step_kernel_sparse<S, NW, MASK, PACKED><<<blocks, kStepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class S, int NW, bool MASK, bool PACKED, int ST, bool GUO, bool SC, bool RL>
static cudaError_t staged_launch(const StepArgs& a, cudaStream_t s);

// One launch per part of a sparse lattice: the rows of plain vectors (the
// unmasked row-chunk kernel over the row list, staged shapes only), the
// list's plain vectors, then the vectors with a link bit or a solid node.
template <class S, int NW, bool PACKED, int ST>
static cudaError_t sparse_parts(const StepArgs& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if constexpr (ST > 0) {
        if (a.nrows > 0) e = staged_launch<S, NW, false, PACKED, ST, false, false, true>(a, s);
    }
    if (e == cudaSuccess && a.ptasks > 0) {
        StepArgs p = a;
        p.vtasks = a.ptasks;
        e = sparse_launch<S, NW, false, PACKED, ST>(p, s);
    }
    if (e == cudaSuccess && a.vtasks > a.ptasks) {
        StepArgs m = a;
        m.vlist = a.vlist + 32LL * a.ptasks;
        m.vinfo = a.vinfo + 32LL * a.ptasks;
        m.vtasks = a.vtasks - a.ptasks;
        e = sparse_launch<S, NW, true, PACKED, ST>(m, s);
    }
    return e;
}

// Persistent grid: as many kStepThreads-thread blocks as fit on the device at once
// (occupancy query, cached per kernel), capped by the work.
template <class S, int NW, bool MASK, bool PACKED, bool GUO, bool SC = false>
static cudaError_t step_launch(const StepArgs& a, cudaStream_t s) {
    static int resident = 0;      // blocks per device, computed once
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_kernel<S, NW, MASK, PACKED, GUO, SC>, kStepThreads, 0);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int wpb = kStepThreads / 32;
    const long long need = (a.ntasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    step_kernel<S, NW, MASK, PACKED, GUO, SC><<<blocks, kStepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class S, int NW, bool MASK, bool PACKED, int ST, bool GUO = false, bool SC = false, bool RL = false>
static cudaError_t staged_launch(const StepArgs& a, cudaStream_t s) {
    constexpr int SW = StageOf<S, NW, MASK>::kWords;
    constexpr int kThreads = staged_threads<S>();
    constexpr int kSmem = (kThreads / 32) * ST * SW * 4;
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel_staged<S, NW, MASK, PACKED, ST, GUO, SC, RL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, step_kernel_staged<S, NW, MASK, PACKED, ST, GUO, SC, RL>, kThreads, kSmem);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int wpb = kThreads / 32;
    const long long ntasks = RL ? (long long)a.nrows * a.chunks : a.ntasks;
    const long long need = (ntasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    step_kernel_staged<S, NW, MASK, PACKED, ST, GUO, SC, RL><<<blocks, kThreads, kSmem, s>>>(a);
    return cudaGetLastError();
}

// M2 forcing: relax constant 9 is set (lattices without solid nodes run it
// on the staged ring in the default shape, the others on direct loads).
__host__ __device__ inline bool uses_guo(const RelaxBoth& r) { return r.d[9] != 0.0; }
__device__ __forceinline__ bool uses_guo_dev(const RelaxBoth& r) { return r.f[9] != 0.0f; }

template <class S, int NW, bool MASK, bool PACKED>
static cudaError_t step_stages(const StepArgs& a, cudaStream_t s) {
    // the Shan-Chen force (lattices without solid nodes) and the M2 terms:
    // the staged ring in the default shape (16-byte vectors, packed pairs,
    // two stages, no solid nodes), else direct-load kernels
    if constexpr (!MASK) {
        const bool guo = uses_guo(a.relax), sc = a.force_kind == 4;
        if constexpr (NW == 4 && (PACKED || sizeof(S) == 8)) {
            if (a.stages == 2 && (guo || sc)) {
                if (sc) return guo ? staged_launch<S, NW, false, PACKED, 2, true, true>(a, s)
                                   : staged_launch<S, NW, false, PACKED, 2, false, true>(a, s);
                return staged_launch<S, NW, false, PACKED, 2, true, false>(a, s);
            }
        }
        if (sc)
            return guo ? step_launch<S, NW, false, PACKED, true, true>(a, s)
                       : step_launch<S, NW, false, PACKED, false, true>(a, s);
    }
    if (uses_guo(a.relax)) return step_launch<S, NW, MASK, PACKED, true>(a, s);
    if constexpr (MASK) {
        if (a.vlist || a.nrows > 0) {
            switch (a.stages) {
                case 0: return sparse_parts<S, NW, PACKED, 0>(a, s);
                case 2: return sparse_parts<S, NW, PACKED, 2>(a, s);
                case 3: return sparse_parts<S, NW, PACKED, 3>(a, s);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (a.stages) {
        case 0: return step_launch<S, NW, MASK, PACKED, false>(a, s);
        case 2: return staged_launch<S, NW, MASK, PACKED, 2>(a, s);
        case 3: return staged_launch<S, NW, MASK, PACKED, 3>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <class S, int NW, bool PACKED>
static cudaError_t step_m(const StepArgs& a, cudaStream_t s) {
    return a.lmask ? step_stages<S, NW, true, PACKED>(a, s) : step_stages<S, NW, false, PACKED>(a, s);
}

// ---------------------------------------------------------------------------
// Batched step: one launch advances every lattice of a batch by one step.
// The tasks of all lattices form one flat list (lattice d owns tasks
// task0[d] .. task0[d+1]-1, row-major chunks); a persistent grid of warps
// walks it.  Each lattice has its own geometry, rates, force and masks
// (a BatchDomain in global memory); `parity` selects which of its two
// population copies is the source.  The launch boundary is the step barrier.
// ---------------------------------------------------------------------------
// The tasks of warp w under the two schedules of the flat task list:
// contiguous (one range per warp, so a warp changes lattice only at lattice
// boundaries) or interleaved (task w + k * nwarps, so the warps sweep the
// batch together as one band, like the single-lattice kernel).  The library
// keeps the task count below 2^31.
struct TaskRange {
    int first, step, end;
    __device__ __forceinline__ TaskRange(int schedule, int ntasks) {
        const int nwarps = gridDim.x * (blockDim.x >> 5);
        const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (schedule) {
            first = w;
            step = nwarps;
            end = ntasks;
        } else {
            first = (int)((long long)w * ntasks / nwarps);
            step = 1;
            end = (int)((long long)(w + 1) * ntasks / nwarps);
        }
    }
};

// A warp's position in the flat task list: task t, its lattice d (tasks up
// to t1 - 1) and the first vector of the task, vector c of row y (rows of
// `nvec` vectors).  Moving on by the warp's task stride stays in integer
// additions while the next task is in the same lattice; only a move to
// another lattice searches and divides.
struct TaskCursor {
    int t = 0, d = -1, t1 = 0;
    int y = 0, c = 0;
    int nvec = 1, dy = 0, dc = 0;     // the stride, 32 vectors per task, as rows and vectors

    __device__ __forceinline__ void locate(const BatchDomain* __restrict__ doms, const int* __restrict__ task0,
                                           int ndom, int ntasks, int task, int step) {
        t = task;
        int t0;
        const int t2 = d >= 0 && d + 2 < ndom ? task0[d + 2] : ntasks;
        if (d >= 0 && t >= t1 && d + 1 < ndom && t < t2) {   // tasks only move forward
            ++d;
            t0 = t1;
            t1 = t2;
        } else {
            int lo = 0, hi = ndom - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (task0[mid] <= t) lo = mid; else hi = mid - 1;
            }
            d = lo;
            t0 = task0[d];
            t1 = d + 1 < ndom ? task0[d + 1] : ntasks;
        }
        nvec = doms[d].a.chunks;
        const long long vstep = 32LL * step, base = 32LL * (t - t0);
        dy = (int)(vstep / nvec);
        dc = (int)(vstep - (long long)dy * nvec);
        y = (int)(base / nvec);
        c = (int)(base - (long long)y * nvec);
    }
    __device__ __forceinline__ void start(const BatchDomain* __restrict__ doms, const int* __restrict__ task0,
                                          int ndom, int ntasks, int task, int step) {
        if (task < ntasks) locate(doms, task0, ndom, ntasks, task, step);
        else t = task;
    }
    // the next task of this warp, t + step (no position past `end`)
    __device__ __forceinline__ void advance(const BatchDomain* __restrict__ doms, const int* __restrict__ task0,
                                            int ndom, int ntasks, int step, int end) {
        const int nt = t + step;
        if (nt >= end) {
            t = nt;
        } else if (nt < t1) {
            t = nt;
            y += dy;
            c += dc;
            if (c >= nvec) {
                c -= nvec;
                ++y;
            }
        } else {
            locate(doms, task0, ndom, ntasks, nt, step);
        }
    }
};

// Which lattices of a batch have solid nodes: none (MM 0: the unmasked path
// only), all (MM 1) or some (MM 2).  With SPLIT (the persistent launch) a
// task runs the masked step when its lattice has solid nodes and its 32
// vectors, from vector c of row y on, reach a row outside [plain_y0,
// plain_y1), the lattice's rows of plain vectors (no link bit, no solid
// node); tasks inside run the unmasked step, the same per-node operations
// without the mask reads and checks (the channels of a sweep: all rows but
// the wall and the two beside it).  256-channel sweep: persistent 0.813 ->
// 0.853 of HBM; the one-launch-per-step kernels, which would carry both
// paths, ran slower with it (0.790 -> 0.748) and keep one path for MM 1.
template <int MM, bool SPLIT>
__device__ __forceinline__ bool task_masked(const StepArgs& a, int y, int c) {
    if constexpr (MM == 0) {
        return false;
    } else if constexpr (!SPLIT) {
        return MM == 1 || a.lmask != nullptr;
    } else {
        if (MM == 2 && a.lmask == nullptr) return false;
        if (y < a.plain_y0) return true;
        const int nvec = a.chunks;
        const int ylast = c + 31 < nvec ? y : y + (c + 31) / nvec;   // row of the last vector
        return ylast >= a.plain_y1;
    }
}

template <class S, int NW, int MM, bool PACKED, bool STAGED, bool GUO, bool SPLIT = false>
__device__ __forceinline__ void batch_chunk(const StepArgs& a, const void* src, void* dst, int y, int c,
                                            int lane, const Coef<typename StepT<S, PACKED>::T>& kc,
                                            const uint32_t* stg) {
    if constexpr (MM != 0) {
        if (task_masked<MM, SPLIT>(a, y, c)) {
            step_chunk<S, NW, true, PACKED, STAGED, GUO, 1>(a, src, dst, y, c, lane, kc, stg);
            return;
        }
    }
    if constexpr (MM != 1 || SPLIT) step_chunk<S, NW, false, PACKED, STAGED, GUO, 1>(a, src, dst, y, c, lane, kc, stg);
}

template <class S, int NW, int MM, bool PACKED, bool GUO>
__global__ void __launch_bounds__(kStepThreads)
batch_step_kernel(const BatchDomain* __restrict__ doms, const int* __restrict__ task0,
                  int ndom, int ntasks, int parity, int schedule) {
    using T = typename StepT<S, PACKED>::T;
    const int lane = threadIdx.x & 31;
    const TaskRange r(schedule, ntasks);
    TaskCursor cc;
    cc.start(doms, task0, ndom, ntasks, r.first, r.step);
    Coef<T> kc;
    int kd = -1;                                 // lattice of kc
    for (; cc.t < r.end; cc.advance(doms, task0, ndom, ntasks, r.step, r.end)) {
        const StepArgs& a = doms[cc.d].a;
        if (cc.d != kd) {
            kc = coef_of<T>(a.relax, a.rho0 * a.scale);
            kd = cc.d;
        }
        const void* src = parity ? a.dst : a.src;
        void* dst = parity ? const_cast<void*>(a.src) : a.dst;
        if (GUO && uses_guo(a.relax))
            batch_chunk<S, NW, MM, PACKED, false, GUO>(a, src, dst, cc.y, cc.c, lane, kc, nullptr);
        else
            batch_chunk<S, NW, MM, PACKED, false, false>(a, src, dst, cc.y, cc.c, lane, kc, nullptr);
    }
}

// Batched step with the shared-memory ring of step_kernel_staged: the issue
// cursor runs ST-1 task strides ahead of the compute cursor; the link word
// of the next task to issue is read one iteration before its issue.
template <class S, int NW, int MM, bool PACKED, int ST>
__global__ void __launch_bounds__(kStepThreads)
batch_step_kernel_staged(const BatchDomain* __restrict__ doms, const int* __restrict__ task0,
                         int ndom, int ntasks, int parity, int schedule) {
    using T = typename StepT<S, PACKED>::T;
    // stage size: with solid nodes anywhere in the batch, the masked layout
    // (its leading offsets are those of the unmasked one)
    constexpr int SW = StageOf<S, NW, MM != 0, 1>::kWords;
    extern __shared__ __align__(16) uint32_t smem_stage[];
    const int lane = threadIdx.x & 31;
    uint32_t* wb = smem_stage + (threadIdx.x >> 5) * ST * SW;
    const TaskRange r(schedule, ntasks);
    const int t_end = r.end, tstep = r.step;
    TaskCursor ci, cc;                           // issue and compute cursors
    ci.start(doms, task0, ndom, ntasks, r.first, r.step);
    cc.start(doms, task0, ndom, ntasks, r.first, r.step);
    // the two cursors' lattice descriptors, copied into this warp's shared
    // memory when a cursor moves to another lattice: fields are read where
    // they are used instead of holding some 30 registers across the loop,
    // which with the compact stage lets four blocks share an SM (measured on
    // the 256-channel sweep: 0.751 -> 0.765 of HBM; the shared copies alone,
    // with the six-slot stage and three blocks, 0.732)
    __shared__ StepArgs sdesc[kStepThreads / 32][2];
    StepArgs& ai = sdesc[threadIdx.x >> 5][0];
    StepArgs& ac = sdesc[threadIdx.x >> 5][1];
    auto fetch = [&](StepArgs& to, int d) {
        static_assert(sizeof(StepArgs) % 8 == 0, "descriptor copied in 8-byte words");
        constexpr int kWords = (int)(sizeof(StepArgs) / 8);
        const unsigned long long* from = reinterpret_cast<const unsigned long long*>(&doms[d].a);
        unsigned long long* dstw = reinterpret_cast<unsigned long long*>(&to);
        __syncwarp();
        for (int k = lane; k < kWords; k += 32) dstw[k] = from[k];
        __syncwarp();
    };
    int aid = -1, acd = -1;
    auto issue = [&](uint32_t* stg, const ChunkMask& cm) {
        const void* src = parity ? ai.dst : ai.src;
        if (task_masked<MM, false>(ai, ci.y, ci.c)) {
            if constexpr (MM != 0) issue_chunk<S, NW, true, 1>(ai, src, ci.y, ci.c, lane, stg, cm);
        } else {
            if constexpr (MM != 1) issue_chunk<S, NW, false, 1>(ai, src, ci.y, ci.c, lane, stg, cm);
        }
    };
    // link word of the issue cursor's chunk (empty without solid nodes)
    auto mask_of = [&]() {
        if (ci.d != aid) {
            fetch(ai, ci.d);
            aid = ci.d;
        }
        ChunkMask cm;
        if constexpr (MM != 0) {
            if (task_masked<MM, false>(ai, ci.y, ci.c)) cm = load_chunk_mask<S, NW, 1>(ai, ci.y, ci.c, lane);
        }
        return cm;
    };
#pragma unroll
    for (int st = 0; st < ST - 1; ++st) {
        if (ci.t < t_end) {
            issue(wb + st * SW, mask_of());
            ci.advance(doms, task0, ndom, ntasks, tstep, t_end);
        }
        cp_async_commit();
    }
    ChunkMask nxt;                              // read one iteration before its issue
    if (ci.t < t_end) nxt = mask_of();
    Coef<T> kc;
    int slot = 0;
    while (cc.t < t_end) {
        cp_async_wait<ST - 2>();
        const int islot = slot == 0 ? ST - 1 : slot - 1;
        if (ci.t < t_end) {
            issue(wb + islot * SW, nxt);
            ci.advance(doms, task0, ndom, ntasks, tstep, t_end);
        }
        cp_async_commit();
        if (ci.t < t_end) nxt = mask_of();
        if (cc.d != acd) {
            fetch(ac, cc.d);
            acd = cc.d;
            kc = coef_of<T>(ac.relax, ac.rho0 * ac.scale);
        }
        const void* src = parity ? ac.dst : ac.src;
        void* dst = parity ? const_cast<void*>(ac.src) : ac.dst;
        batch_chunk<S, NW, MM, PACKED, true, false>(ac, src, dst, cc.y, cc.c, lane, kc, wb + slot * SW);
        cc.advance(doms, task0, ndom, ntasks, tstep, t_end);
        slot = slot + 1 == ST ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

template <class S, int NW, int MM, bool PACKED, int ST>
static cudaError_t batch_launch_staged(const BatchLaunch& b, cudaStream_t s) {
    constexpr int SW = StageOf<S, NW, MM != 0, 1>::kWords;
    constexpr int kSmem = (kStepThreads / 32) * ST * SW * 4;
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_step_kernel_staged<S, NW, MM, PACKED, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, batch_step_kernel_staged<S, NW, MM, PACKED, ST>, kStepThreads, kSmem);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int wpb = kStepThreads / 32;
    const int need = (b.ntasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    batch_step_kernel_staged<S, NW, MM, PACKED, ST><<<blocks, kStepThreads, kSmem, s>>>(
        b.doms, b.task0, b.ndom, b.ntasks, b.parity, b.schedule);
    return cudaGetLastError();
}

template <class S, int NW, int MM, bool PACKED, bool GUO>
static cudaError_t batch_launch(const BatchLaunch& b, cudaStream_t s) {
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, batch_step_kernel<S, NW, MM, PACKED, GUO>, kStepThreads, 0);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int wpb = kStepThreads / 32;
    const int need = (b.ntasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(need < resident ? need : resident);
    batch_step_kernel<S, NW, MM, PACKED, GUO><<<blocks, kStepThreads, 0, s>>>(
        b.doms, b.task0, b.ndom, b.ntasks, b.parity, b.schedule);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent batched steps: one cooperative launch advances every lattice by
// nsteps steps.  The streaming warps split the flat task list into
// contiguous ranges (every active warp has at least one task); between
// steps a warp waits only for the lattices it works on: a lattice's counter
// counts the warps that finished their tasks of it at the current step, and
// a warp issues the copies of lattice d for step s only once d's counter has
// reached s times the number of warps that work on d.  That wait covers both
// the reads of step s (they need step s - 1 complete) and the writes of
// step s (they overwrite what step s - 1 read).  The dependencies point only
// to earlier steps or to earlier tasks of the same step, so with every
// block resident (cooperative launch) the waits cannot form a cycle; each
// one still polls a bounded number of times, and a warp that gives up
// records it in the status word and leaves (the others then give up too).
// Lattices small enough to fit twice in a block's shared memory are held
// there for the whole launch, one block each.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The contiguous split of T tasks over A active warps: first task of warp w,
// and the warp that holds task t.
__device__ __forceinline__ int split_first(int w, int T, int A) { return (int)((long long)w * T / A); }
__device__ __forceinline__ int split_warp(int t, int T, int A) {
    return (int)(((long long)(t + 1) * A - 1) / T);
}

// Lane 0 polls the counter until it reaches target (bounded), the warp
// follows; false when it gave up or another warp had given up.
__device__ __forceinline__ bool wait_counter(const BatchLaunch& p, const unsigned* ctr, unsigned target,
                                             int lane) {
    int ok = 1;
    if (lane == 0) {
        unsigned polls = 0;
        while (ld_acquire_u32(ctr) < target) {
            if (ld_relaxed_s32(p.status) != 0) { ok = 0; break; }
            if (polls++ >= p.spin_limit) {
                atomicCAS(p.status, 0, 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (ok) __threadfence();
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// One lattice held in this block's shared memory (two copies of its state)
// for nsteps steps: the per-node operations of the streaming step (pull
// with halfway bounce-back, Eq. 10 and Sec. 4A; collision, Eq. 11-15), one
// node per thread, in the same arithmetic, so the bits are those of the
// streaming step.  Populations stay in the storage format; the collision
// works in scaled deviations as in step_chunk.
template <class S>
__device__ void resident_steps(const StepArgs& a, int parity, int nsteps, uint32_t* smem) {
    using C = typename Fmt<S>::C;
    using R = typename std::conditional<sizeof(S) == 8, unsigned long long,
              typename std::conditional<sizeof(S) == 4, uint32_t, unsigned short>::type>::type;
    const int nx = a.geo.nx, ny = a.geo.ny, pitch = a.geo.pitch;
    const long long plane = a.geo.plane;
    const int n = nx * ny;
    R* b0 = reinterpret_cast<R*>(smem);
    R* b1 = b0 + 9 * n;
    const R* gsrc = static_cast<const R*>(parity ? a.dst : a.src);
    for (int k = threadIdx.x; k < 9 * n; k += blockDim.x) {
        const int i = k / n, q = k - i * n, y = q / nx, x = q - y * nx;
        b0[k] = gsrc[i * plane + (long long)y * pitch + x];
    }
    __syncthreads();
    const Coef<C> kc = coef_of<C>(a.relax, a.rho0 * a.scale);
    const bool guo = uses_guo_dev(a.relax);
    const C* Fa = static_cast<const C*>(a.force);
    const C sc = scale_of<C>(a);
    for (int st = 0; st < nsteps; ++st) {
        const R* from = (st & 1) ? b1 : b0;
        R* to = (st & 1) ? b0 : b1;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int y = q / nx, x = q - y * nx;
            const long long gq = (long long)y * pitch + x;
            uint32_t links = 0u;
            bool solid = false;
            if (a.lmask) {
                links = a.lmask[gq];
                solid = (a.sbits[gq >> 3] >> (gq & 7)) & 1u;
            }
            if (solid) {
#pragma unroll
                for (int i = 0; i < 9; ++i) to[i * n + q] = R(0);
                continue;
            }
            C g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                R v;
                if (i > 0 && ((links >> (i - 1)) & 1u)) {
                    v = from[opp_of(i) * n + q];                 // halfway bounce-back
                } else {
                    int xs = x - ex_of(i), ys = y - ey_of(i);
                    xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
                    v = from[i * n + ys * nx + xs];
                }
                uint32_t w4[4] = {0u, 0u, 0u, 0u};
                if constexpr (sizeof(S) == 8) {
                    w4[0] = (uint32_t)v;
                    w4[1] = (uint32_t)((unsigned long long)v >> 32);
                } else {
                    w4[0] = (uint32_t)v;
                }
                g[i] = Fmt<S>::get(w4, 0);
            }
            C Fx, Fy;
            if (a.force_kind == 1) {
                Fx = Fa[2 * y] * sc;
                Fy = Fa[2 * y + 1] * sc;
            } else if (a.force_kind == 2 || a.force_kind == 3) {
                const long long k2 = 2 * ((a.force_kind == 2 ? 0 : (long long)y * nx) + x);
                Fx = Fa[k2] * sc;
                Fy = Fa[k2 + 1] * sc;
            } else {
                Fx = fxs_of<C>(a);
                Fy = fys_of<C>(a);
            }
            if (guo)
                collide<C, true>(g, Fx, Fy, kc);
            else
                collide<C, false>(g, Fx, Fy, kc);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                uint32_t w4[4] = {0u, 0u, 0u, 0u};
                if constexpr (sizeof(S) == 8) {
                    Fmt<S>::set(w4, 0, g[i]);
                    to[i * n + q] = ((unsigned long long)w4[1] << 32) | w4[0];
                } else {
                    Fmt<S>::set(w4, 0, g[i]);
                    to[i * n + q] = (R)w4[0];
                }
            }
        }
        __syncthreads();
    }
    const R* fin = (nsteps & 1) ? b1 : b0;
    R* gdst = static_cast<R*>((parity ^ (nsteps & 1)) ? a.dst : const_cast<void*>(a.src));
    for (int k = threadIdx.x; k < 9 * n; k += blockDim.x) {
        const int i = k / n, q = k - i * n, y = q / nx, x = q - y * nx;
        gdst[i * plane + (long long)y * pitch + x] = fin[k];
    }
    __syncthreads();                            // the block's next lattice reuses the memory
}

// Four blocks of the FP32 batch kernels share an SM (124-128 registers; per
// warp the compact stage's two slots and two lattice descriptors in shared
// memory, plus 1 KB the SM reserves per block, within its 228 KB): a larger
// descriptor or stage leaves room for three (measured when StepArgs grew by
// 16 bytes: 256-channel sweep 0.86 -> 0.83 of HBM).
static_assert(4 * ((kStepThreads / 32) * (2 * StageOf<float, 4, true, 1>::kWords * 4 + 2 * (int)sizeof(StepArgs)) +
                   1024) <= 228 * 1024,
              "four FP32 batch blocks per SM");

template <class S, int NW, int MM, bool PACKED, int ST>
__global__ void __launch_bounds__(kStepThreads) batch_persist_kernel(const BatchLaunch p) {
    using T = typename StepT<S, PACKED>::T;
    constexpr int SW = StageOf<S, NW, MM != 0, 1>::kWords;
    extern __shared__ __align__(16) uint32_t smem_stage[];
    if ((int)blockIdx.x < p.res_blocks) {
        for (int k = p.res_first[blockIdx.x]; k < p.res_first[blockIdx.x + 1]; ++k)
            resident_steps<S>(p.doms[p.ndom + k].a, p.parity, p.nsteps, smem_stage);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int nw = (gridDim.x - p.res_blocks) * wpb;
    const int NT = p.ntasks;
    const int A = nw < NT ? nw : NT;                 // active warps: at least one task each
    const int w = (blockIdx.x - p.res_blocks) * wpb + (threadIdx.x >> 5);
    if (w >= A) return;
    const int t_first = split_first(w, NT, A), t_end = split_first(w + 1, NT, A);
    uint32_t* wb = smem_stage + (threadIdx.x >> 5) * ST * SW;
    __shared__ StepArgs sdesc[kStepThreads / 32][2];
    StepArgs& ai = sdesc[threadIdx.x >> 5][0];
    StepArgs& ac = sdesc[threadIdx.x >> 5][1];
    auto fetch = [&](StepArgs& to, int d) {
        constexpr int kWords = (int)(sizeof(StepArgs) / 8);
        const unsigned long long* from = reinterpret_cast<const unsigned long long*>(&p.doms[d].a);
        unsigned long long* dstw = reinterpret_cast<unsigned long long*>(&to);
        __syncwarp();
        for (int k = lane; k < kWords; k += 32) dstw[k] = from[k];
        __syncwarp();
    };
    if (p.delay_ns != 0u && w == 0) {              // test hook: a late first warp
        if (lane == 0)
            for (unsigned left = p.delay_ns; left > 0u;) {
                const unsigned d = left < 100000u ? left : 100000u;
                __nanosleep(d);
                left -= d;
            }
        __syncwarp();
    }
    int aid = -1, acd = -1;
    Coef<T> kc;
    for (int s = 0; s < p.nsteps; ++s) {
        const int parity = p.parity ^ (s & 1);
        TaskCursor ci, cc;                         // issue and compute cursors
        ci.start(p.doms, p.task0, p.ndom, NT, t_first, 1);
        cc.start(p.doms, p.task0, p.ndom, NT, t_first, 1);
        int ready = -1;                            // lattice cleared for step s
        bool ok = true;
        // before the first copy of lattice d at step s: all its warps are
        // through step s - 1
        auto gate = [&](int d) -> bool {
            if (d == ready) return true;
            ready = d;
            if (s == 0) return true;
            const int lo = __ldg(p.task0 + d);
            const int hi = d + 1 < p.ndom ? __ldg(p.task0 + d + 1) : NT;
            const unsigned workers = (unsigned)(split_warp(hi - 1, NT, A) - split_warp(lo, NT, A) + 1);
            return wait_counter(p, p.done + d, (unsigned)s * workers, lane);
        };
        auto mask_of = [&]() {
            if (ci.d != aid) {
                fetch(ai, ci.d);
                aid = ci.d;
            }
            ChunkMask cm;
            if constexpr (MM != 0) {
                if (task_masked<MM, true>(ai, ci.y, ci.c)) cm = load_chunk_mask<S, NW, 1>(ai, ci.y, ci.c, lane);
            }
            return cm;
        };
        auto issue = [&](uint32_t* stg, const ChunkMask& cm) {
            const void* src = parity ? ai.dst : ai.src;
            if (task_masked<MM, true>(ai, ci.y, ci.c)) {
                if constexpr (MM != 0) issue_chunk<S, NW, true, 1>(ai, src, ci.y, ci.c, lane, stg, cm);
            } else {
                issue_chunk<S, NW, false, 1>(ai, src, ci.y, ci.c, lane, stg, cm);
            }
        };
#pragma unroll
        for (int st = 0; st < ST - 1; ++st) {
            if (ok && ci.t < t_end) {
                const ChunkMask cm = mask_of();
                ok = gate(ci.d);
                if (ok) {
                    issue(wb + st * SW, cm);
                    ci.advance(p.doms, p.task0, p.ndom, NT, 1, t_end);
                }
            }
            cp_async_commit();
        }
        ChunkMask nxt;
        if (ok && ci.t < t_end) nxt = mask_of();
        int slot = 0;
        while (ok && cc.t < t_end) {
            cp_async_wait<ST - 2>();
            const int islot = slot == 0 ? ST - 1 : slot - 1;
            if (ci.t < t_end) {
                ok = gate(ci.d);
                if (!ok) break;
                issue(wb + islot * SW, nxt);
                ci.advance(p.doms, p.task0, p.ndom, NT, 1, t_end);
            }
            cp_async_commit();
            if (ci.t < t_end) nxt = mask_of();
            if (cc.d != acd) {
                fetch(ac, cc.d);
                acd = cc.d;
                kc = coef_of<T>(ac.relax, ac.rho0 * ac.scale);
            }
            const void* src = parity ? ac.dst : ac.src;
            void* dst = parity ? const_cast<void*>(ac.src) : ac.dst;
            batch_chunk<S, NW, MM, PACKED, true, false, true>(ac, src, dst, cc.y, cc.c, lane, kc, wb + slot * SW);
            const int dprev = cc.d;
            cc.advance(p.doms, p.task0, p.ndom, NT, 1, t_end);
            if (cc.t >= t_end || cc.d != dprev) {  // this warp's tasks of the lattice are stored
                __syncwarp();
                if (lane == 0) red_release_add_u32(p.done + dprev, 1u);
            }
            slot = slot + 1 == ST ? 0 : slot + 1;
        }
        cp_async_wait<0>();
        if (!ok) return;
    }
}

template <class S, int NW, int MM, bool PACKED, int ST>
static cudaError_t batch_launch_persist(const BatchLaunch& b, cudaStream_t s) {
    constexpr int SW = StageOf<S, NW, MM != 0, 1>::kWords;
    constexpr int kSmem = (kStepThreads / 32) * ST * SW * 4;
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batch_persist_kernel<S, NW, MM, PACKED, ST>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, batch_persist_kernel<S, NW, MM, PACKED, ST>, kStepThreads, kSmem);
        if (e != cudaSuccess) return e;
        resident = sms * (per_sm > 0 ? per_sm : 1);
    }
    if (b.nsteps < 1) return cudaSuccess;
    if (b.res_blocks < 0 || b.res_blocks >= resident) return cudaErrorInvalidValue;
    const int wpb = kStepThreads / 32;
    const long long want = b.res_blocks + (b.ntasks + wpb - 1) / wpb;
    const unsigned blocks = (unsigned)(want < resident ? want : resident);
    cudaError_t e = cudaMemsetAsync(b.done, 0, (size_t)(b.ndom > 0 ? b.ndom : 1) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kStepThreads);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every block resident at once
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_persist_kernel<S, NW, MM, PACKED, ST>, b);
}

template <class S, int NW, int MM, bool PACKED>
static cudaError_t batch_stages(const BatchLaunch& b, cudaStream_t s) {
    if (b.persist) {
        switch (b.stages) {
            case 2: return batch_launch_persist<S, NW, MM, PACKED, 2>(b, s);
            case 3: return batch_launch_persist<S, NW, MM, PACKED, 3>(b, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (b.stages) {
        case 0: return batch_launch<S, NW, MM, PACKED, false>(b, s);
        case 2: return batch_launch_staged<S, NW, MM, PACKED, 2>(b, s);
        case 3: return batch_launch_staged<S, NW, MM, PACKED, 3>(b, s);
    }
    return cudaErrorInvalidValue;
}

template <class S, int NW, bool PACKED>
static cudaError_t batch_shape(const BatchLaunch& b, cudaStream_t s) {
    // a batch with any M2 lattice runs on the direct-load kernel with both
    // chunk paths
    if (b.guo) return batch_launch<S, NW, 2, PACKED, true>(b, s);
    switch (b.mask_mode) {
        case 0: return batch_stages<S, NW, 0, PACKED>(b, s);
        case 1: return batch_stages<S, NW, 1, PACKED>(b, s);
        case 2: return batch_stages<S, NW, 2, PACKED>(b, s);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_batch_format(const BatchLaunch& b, cudaStream_t s) {
    if constexpr (sizeof(S) == 8) {
        return batch_shape<S, 4, false>(b, s);
    } else {
        if (b.vec_bytes == 16)
            return b.packed ? batch_shape<S, 4, true>(b, s) : batch_shape<S, 4, false>(b, s);
        return b.packed ? batch_shape<S, 2, true>(b, s) : batch_shape<S, 2, false>(b, s);
    }
}

// Every launch shape of one storage format (see clbm_set_tuning).
template <class S>
static cudaError_t launch_step_format(const StepArgs& a, cudaStream_t s) {
    if constexpr (sizeof(S) == 8) {
        return step_m<S, 4, false>(a, s);
    } else {
        if (a.vec_bytes == 16)
            return a.packed ? step_m<S, 4, true>(a, s) : step_m<S, 4, false>(a, s);
        return a.packed ? step_m<S, 2, true>(a, s) : step_m<S, 2, false>(a, s);
    }
}

}  // namespace clbm
