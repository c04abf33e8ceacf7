// clbm_host.h -- host-side helpers shared by the single-lattice API
// (clbm_api.cu) and the batch API (clbm_batch.cu): argument checks, the
// relaxation constants of Eq. 7, row pitches, the bounce-back link bits and
// solid bitmap, and the force array in the compute type.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_device.cuh"
#include "clbm_internal.h"

namespace clbm {

inline bool all_finite(const double* p, size_t n) {
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(p[k])) return false;
    return true;
}

// number of FP64 values of a force array of the given layout
inline size_t force_values(int kind, int nx, int ny) {
    return kind == CLBM_FORCE_ROWS         ? 2 * (size_t)ny
           : kind == CLBM_FORCE_COLUMNS    ? 2 * (size_t)nx
           : kind == CLBM_FORCE_FIELD      ? 2 * (size_t)nx * ny
           : kind == CLBM_FORCE_SHAN_CHEN  ? 3   // G, psi0, rho0
                                           : 0;
}

// Checks shared by clbm_create and clbm_batch_create (see include/clbm.h).
inline int check_lattice_args(int nx, int ny, const double* rates, int force_kind,
                              const double* force, double fx, double fy, int format) {
    if (nx < 2 || ny < 2 || !rates) return CLBM_ERR_ARG;
    if ((long long)nx * ny > (1LL << 36)) return CLBM_ERR_ARG;
    if ((long long)ny * ((nx + 63) / 64) >= (1LL << 31)) return CLBM_ERR_ARG;   // task count
    if (format < CLBM_FP64 || format > CLBM_BF16) return CLBM_ERR_ARG;
    for (int k = 0; k < 9; ++k)
        if (!(rates[k] > 0.0 && rates[k] < 2.0)) return CLBM_ERR_ARG;
    if (rates[1] != rates[2] || rates[4] != rates[5] || rates[6] != rates[7]) return CLBM_ERR_ARG;
    if (force_kind < CLBM_FORCE_UNIFORM || force_kind > CLBM_FORCE_SHAN_CHEN) return CLBM_ERR_ARG;
    if (force_kind != CLBM_FORCE_UNIFORM && !force) return CLBM_ERR_ARG;
    if (!std::isfinite(fx) || !std::isfinite(fy)) return CLBM_ERR_ARG;
    const size_t nforce = force_values(force_kind, nx, ny);
    if (nforce && !all_finite(force, nforce)) return CLBM_ERR_ARG;
    if (force_kind == CLBM_FORCE_SHAN_CHEN && !(force[1] > 0.0)) return CLBM_ERR_ARG;   // psi0 > 0
    return CLBM_OK;
}

// Eq. 7 rates (s0, s1, s1, sb, s2, s2, s3, s3, s4) and the forcing scheme
// (clbm_forcing) -> the collision's constants.  The schemes differ only in
// the forcing moments: the consistent one (Eq. 12, 14) weights C6, C7 by
// (1 - s3/2); M1 (Eq. 17-19) has no third-order forcing moments; M2 (Eq. 21)
// weights Guo's moments by (1 - s2/2), so k~*_10 = (1 + s1 - s2) Fx / 2.
inline void relax_constants(const double* s, int scheme, RelaxBoth& r) {
    double f3 = (1.0 - 0.5 * s[6]) / 3.0, g1 = 0.5, c2 = 0.0, m2 = 0.0;
    if (scheme == CLBM_FORCING_M1) f3 = 0.0;
    if (scheme == CLBM_FORCING_M2) {
        f3 = (1.0 - 0.5 * s[4]) / 3.0;
        g1 = 0.5 * (1.0 + s[1] - s[4]);
        c2 = 1.0 - 0.5 * s[4];
        m2 = 1.0;
    }
    const double v[10] = {1.0 - s[3], 1.0 - s[4], 1.0 - s[6], 1.0 - s[8],
                          s[3] * 2.0 / 3.0, s[8] / 9.0, f3, g1, c2, m2};
    for (int k = 0; k < 10; ++k) {
        r.d[k] = v[k];
        r.f[k] = (float)v[k];
    }
}

// The fields of StepArgs derived from fx, fy, scale and sc_g (the same
// IEEE operations the device would do, once per launch instead of per
// chunk).
inline void derive_args(StepArgs& a) {
    a.fxs_d = a.fx * a.scale;
    a.fys_d = a.fy * a.scale;
    a.scale_f = (float)a.scale;
    a.fxs_f = (float)a.fxs_d;
    a.fys_f = (float)a.fys_d;
    a.sc_g_f = (float)a.sc_g;
}

// stored row length in elements: rows start on 128-byte lines
inline int row_pitch(int nx, int format) {
    const int align = 128 / element_size(format);
    return (nx + align - 1) / align * align;
}

// Link bits (bit i-1 of lmask[y*pitch + x]: node x - e_i solid, periodic)
// and the solid bitmap (bit q & 7 of sbits[q >> 3], q = y*pitch + x);
// padding columns are solid with every link bit set.  The bitmap carries 16
// spare bytes: the staged kernel copies the aligned 4-byte word holding a
// node's flag.  Returns the number of solid nodes.
inline long long build_solid_masks(const uint8_t* solid, int nx, int ny, int pitch,
                                   std::vector<uint8_t>& lmask, std::vector<uint8_t>& sbits) {
    long long nsolid = 0;
    for (long long p = 0; p < (long long)nx * ny; ++p) nsolid += solid[p] != 0;
    const size_t cells = (size_t)pitch * ny;
    lmask.assign(cells, 0xFF);
    sbits.assign((cells + 7) / 8 + 16, 0);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < pitch; ++x) {
            const size_t q = (size_t)y * pitch + x;
            uint8_t b = 0xFF;
            bool is_solid = true;
            if (x < nx) {
                is_solid = solid[(size_t)y * nx + x] != 0;
                b = 0;
                for (int i = 1; i < 9; ++i) {
                    const int xs = ((x - ex_of(i)) % nx + nx) % nx;
                    const int ys = ((y - ey_of(i)) % ny + ny) % ny;
                    if (solid[(size_t)ys * nx + xs]) b |= (uint8_t)(1u << (i - 1));
                }
            }
            lmask[q] = b;
            if (is_solid) sbits[q >> 3] |= (uint8_t)(1u << (q & 7));
        }
    }
    return nsolid;
}

// The bounce-back plan of one vector of a sparse list: the word that the
// sparse step reads beside the list entry, in place of working it out from
// the link bits at every step (Sec. 4A's halfway bounce-back).  Vector v of
// row y holds nodes x = V v .. V v + V - 1 (V <= 8); nodes past the row end
// count as solid with every link bit set, as in build_solid_masks.
//   bits 0-7    solid flag of node j in bit j
//   bits 8-10   the source rows of e_y = -1, 0, +1 (rows y + 1, y, y - 1)
//               are solid under all V nodes
//   bits 11-16  own vectors of the compact stage held in plane slots: bit
//               own_slot(i) where link i bounces at a fluid node and its
//               source row is all solid (so the plane slot is free)
//   bits 17-22  the other own vectors that the bounce-back reads (bit
//               own_slot(i)); with bits 11-16, the links 2, 4, 5, 6, 7, 8
//               that bounce at some fluid node
//   bits 23-24  links 1 and 3 bounce at some fluid node
//   bits 25-27  the left neighbour element of planes 1, 5, 8 is used: node 0
//               is fluid and the link does not bounce there
//   bits 28-30  the right neighbour element of planes 3, 6, 7 is used (at
//               the vector's last node inside the row)
//   bit 31      the vector is not plain (a solid node or a link bit)
// (the shifts are kInfo* in clbm_internal.h)
// Link bytes of row y (bit i-1 of out[x]: the pull source (x - e_ix,
// y - e_iy) of node x is solid, periodic), as build_solid_masks builds them.
inline void row_links(const uint8_t* solid, int nx, int ny, int y, uint8_t* out) {
    const uint8_t* rows[3] = {solid + (size_t)((y + 1) % ny) * nx, solid + (size_t)y * nx,
                              solid + (size_t)((y + ny - 1) % ny) * nx};   // by e_y + 1: rows y+1, y, y-1
    for (int x = 0; x < nx; ++x) {
        const int xl = x == 0 ? nx - 1 : x - 1, xr = x == nx - 1 ? 0 : x + 1;
        uint32_t b = 0;
        for (int i = 1; i < 9; ++i) {
            const uint8_t* r = rows[ey_of(i) + 1];
            const int xs = ex_of(i) > 0 ? xl : ex_of(i) < 0 ? xr : x;
            if (r[xs]) b |= 1u << (i - 1);
        }
        out[x] = (uint8_t)b;
    }
}

// The info word of vector v from the link bytes (`links`, row_links) and
// solid flags (`solid_row`) of its row.
inline uint32_t vector_info_row(const uint8_t* links, const uint8_t* solid_row, int nx, int v, int V) {
    uint32_t sflag = 0, all = 0xff, any_link = 0, bounce = 0, link[8] = {};
    for (int j = 0; j < V; ++j) {
        const int x = v * V + j;
        const uint32_t b = x < nx ? links[x] : 0xffu;
        const bool is_solid = x >= nx || solid_row[x] != 0;
        link[j] = b;
        all &= b;
        any_link |= b;
        if (is_solid) sflag |= 1u << j;
        else bounce |= b;                       // links that bounce at fluid nodes
    }
    const bool row_solid[3] = {((all >> 3) & 1u) != 0, sflag == (1u << V) - 1u, ((all >> 1) & 1u) != 0};
    uint32_t need = 0, cover = 0;
    for (int i = 2; i < 9; ++i) {
        if (i == 3) continue;
        if ((bounce >> (i - 1)) & 1u) need |= 1u << own_slot(i);
        if (row_solid[ey_of(i) + 1]) cover |= 1u << own_slot(i);
    }
    uint32_t w = sflag;
    for (int r = 0; r < 3; ++r)
        if (row_solid[r]) w |= 1u << (kInfoRowShift + r);
    w |= (cover & need) << kInfoCoverShift;
    w |= (need & ~cover) << kInfoRestShift;
    if (bounce & 1u) w |= 1u << kInfoBounce1;
    if ((bounce >> 2) & 1u) w |= 1u << kInfoBounce3;
    // neighbour elements: node 0 on the left, the last node inside the row
    // on the right
    const int jr = std::min(V - 1, nx - 1 - v * V);
    const int left[3] = {1, 5, 8}, right[3] = {3, 6, 7};
    for (int k = 0; k < 3; ++k) {
        if (!(sflag & 1u) && !((link[0] >> (left[k] - 1)) & 1u)) w |= 1u << (kInfoLeftShift + k);
        if (!((sflag >> jr) & 1u) && !((link[jr] >> (right[k] - 1)) & 1u)) w |= 1u << (kInfoRightShift + k);
    }
    if (sflag != 0 || any_link != 0) w |= kInfoNotPlain;
    return w;
}

// The info word of vector v of row y from the solid array alone.
inline uint32_t vector_info(const uint8_t* solid, int nx, int ny, int y, int v, int V) {
    std::vector<uint8_t> links(nx);
    row_links(solid, nx, ny, y, links.data());
    return vector_info_row(links.data(), solid + (size_t)y * nx, nx, v, V);
}

// Rows with no solid node within one step (rows r - 1, r, r + 1,
// periodic): their vectors have no link bit and no solid node.
inline std::vector<uint8_t> plain_rows(const uint8_t* solid, int nx, int ny) {
    std::vector<uint8_t> has(ny, 0), plain(ny, 0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx && !has[y]; ++x) has[y] = solid[(size_t)y * nx + x] != 0;
    for (int y = 0; y < ny; ++y) plain[y] = !has[(y + ny - 1) % ny] && !has[y] && !has[(y + 1) % ny];
    return plain;
}

// The longest run of plain rows [y0, y1) (plain_rows); y0 = y1 = 0 when
// there is none.
inline void plain_row_range(const uint8_t* solid, int nx, int ny, int& y0, int& y1) {
    const std::vector<uint8_t> rows = plain_rows(solid, nx, ny);
    y0 = y1 = 0;
    int run0 = 0;
    for (int y = 0; y <= ny; ++y) {
        const bool plain = y < ny && rows[y];
        if (!plain) {
            if (y - run0 > y1 - y0) {
                y0 = run0;
                y1 = y;
            }
            run0 = y + 1;
        }
    }
}

// FP64 force values -> bytes of the compute type of `format`
inline void force_in_compute_type(const double* force, size_t n, int format,
                                  std::vector<unsigned char>& out) {
    if (format == CLBM_FP64) {
        out.resize(n * sizeof(double));
        std::memcpy(out.data(), force, n * sizeof(double));
    } else {
        out.resize(n * sizeof(float));
        float* f = reinterpret_cast<float*>(out.data());
        for (size_t k = 0; k < n; ++k) f[k] = (float)force[k];
    }
}

// FP16 run scale: deviations are stored times 2^k so the largest sits near
// 2^11 (32x headroom below the FP16 maximum), assuming at least 2^-6 so
// that a quiet start leaves room for the flow to develop.
inline int fp16_scale_exponent(double max_dev) {
    const double mx = std::fmax(max_dev, std::ldexp(1.0, -6));
    const int k = (int)std::floor(std::log2(2048.0 / mx));
    return k < 0 ? 0 : (k > 40 ? 40 : k);
}

}  // namespace clbm
