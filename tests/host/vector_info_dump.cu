// Test harness (host only): prints the sparse list's info word of every
// vector of a lattice, as vector_info in clbm_host.h builds it, so that a
// CPU test can check each field against the solid array directly.
// Usage: vector_info_dump NX NY V SOLID_FILE   (SOLID_FILE: NX*NY bytes,
// row-major, nonzero = solid).  Output: one hexadecimal word per line, for
// rows y = 0 .. NY-1 and vectors v = 0 .. ceil(NX / V) - 1.  With V = 0 it
// prints plain_row_range's two rows (the batch's rows of plain vectors) and
// then plain_rows' flag of every row (the sparse lattices' row list); with
// V = -1, each node's link byte from build_solid_masks and from row_links.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1705_11092_gb300/csrc/clbm_host.h"

int main(int argc, char** argv) {
    if (argc != 5) return 2;
    const int nx = std::atoi(argv[1]), ny = std::atoi(argv[2]), V = std::atoi(argv[3]);
    if (nx < 1 || ny < 1 || V < -1 || V > 8) return 2;
    std::vector<uint8_t> solid((size_t)nx * ny);
    FILE* f = std::fopen(argv[4], "rb");
    if (!f) return 3;
    const size_t got = std::fread(solid.data(), 1, solid.size(), f);
    std::fclose(f);
    if (got != solid.size()) return 3;
    if (V == -1) {       // link bytes: build_solid_masks (x < nx), then row_links
        std::vector<uint8_t> lm, sb, row(nx);
        const int pitch = (nx + 31) / 32 * 32;       // rows padded as for FP32
        clbm::build_solid_masks(solid.data(), nx, ny, pitch, lm, sb);
        for (int y = 0; y < ny; ++y) {
            clbm::row_links(solid.data(), nx, ny, y, row.data());
            for (int x = 0; x < nx; ++x) std::printf("%02x%02x ", lm[(size_t)y * pitch + x], row[x]);
            std::printf("\n");
        }
        return 0;
    }
    if (V == 0) {
        int y0 = -1, y1 = -1;
        clbm::plain_row_range(solid.data(), nx, ny, y0, y1);
        std::printf("%d %d\n", y0, y1);
        const std::vector<uint8_t> rows = clbm::plain_rows(solid.data(), nx, ny);
        for (int y = 0; y < ny; ++y) std::printf("%d", rows[y] ? 1 : 0);
        std::printf("\n");
        return 0;
    }
    const int nvec = (nx + V - 1) / V;
    for (int y = 0; y < ny; ++y)
        for (int v = 0; v < nvec; ++v)
            std::printf("%08x\n", clbm::vector_info(solid.data(), nx, ny, y, v, V));
    return 0;
}
