// Host check of the library's cell numbering (row_pos, cell_index, cell_coords in the internal
// header): for a range of grids and block heights the row numbering is a bijection onto
// [0, n_y n_z) that follows the order (z / kz, y, z % kz), cell_index puts x fastest within a
// row, and cell_coords inverts cell_index.  A few positions are also pinned to values worked out
// by hand from that order.  Runs on the host only; prints "bad 0" when every check holds.
#include <cstdio>
#include <vector>

#include "gbmd_internal.cuh"

using gbmd::Rep;

static Rep grid(int nx, int ny, int nz, int kz)
{
    Rep R{};
    R.nc[0] = nx;
    R.nc[1] = ny;
    R.nc[2] = nz;
    R.kz = kz;
    R.cell0 = 11;
    return R;
}

int main()
{
    int bad = 0;
    long checked = 0;
    const int grids[][3] = {{3, 3, 3}, {4, 5, 7}, {9, 3, 10}, {5, 8, 3}, {13, 6, 17}, {112, 112, 112}, {7, 1023, 9}};
    for (const auto& g : grids) {
        for (int kz = 1; kz <= 16; kz *= 2) {
            const Rep R = grid(g[0], g[1], g[2], kz);
            std::vector<int> seen(size_t(g[1]) * g[2], 0);
            int prev_key = -1, prev_pos = -1;
            // visit rows in the order (z / kz, y, z % kz): their positions must be 0, 1, 2, ...
            for (int zb = 0; zb * kz < g[2]; ++zb)
                for (int y = 0; y < g[1]; ++y)
                    for (int z = zb * kz; z < zb * kz + kz && z < g[2]; ++z) {
                        const int p = gbmd::row_pos(R, y, z);
                        ++checked;
                        if (p != prev_pos + 1) ++bad;
                        prev_pos = p;
                        if (p < 0 || p >= g[1] * g[2]) { ++bad; continue; }
                        seen[p] += 1;
                        const int key = (zb * g[1] + y) * kz + (z - zb * kz);
                        if (key <= prev_key) ++bad;
                        prev_key = key;
                        const int xs[3] = {0, g[0] / 2, g[0] - 1};
                        for (int cx : xs) {
                            const int c = gbmd::cell_index(R, cx, y, z);
                            if (c != R.cell0 + p * g[0] + cx) ++bad;
                            int ax, ay, az;
                            gbmd::cell_coords(R, c - R.cell0, ax, ay, az);
                            if (ax != cx || ay != y || az != z) ++bad;
                        }
                    }
            for (int v : seen)
                if (v != 1) ++bad;
        }
    }
    // by hand: n = (4, 5, 7), kz = 4: block 0 holds planes 0-3 (20 rows), block 1 planes 4-6
    {
        const Rep R = grid(4, 5, 7, 4);
        if (gbmd::row_pos(R, 0, 0) != 0) ++bad;              // first row of block 0
        if (gbmd::row_pos(R, 0, 3) != 3) ++bad;              // y = 0, z % 4 = 3
        if (gbmd::row_pos(R, 1, 0) != 4) ++bad;              // y = 1 starts after the 4 planes of y = 0
        if (gbmd::row_pos(R, 4, 3) != 19) ++bad;             // last row of block 0
        if (gbmd::row_pos(R, 0, 4) != 20) ++bad;             // block 1 starts after 20 rows
        if (gbmd::row_pos(R, 2, 5) != 27) ++bad;             // 20 + 2 * 3 (3 planes in block 1) + 1
        if (gbmd::cell_index(R, 3, 2, 5) != 11 + 27 * 4 + 3) ++bad;
        const Rep P = grid(4, 5, 7, 1);                      // kz = 1: the plain (z, y) order
        if (gbmd::row_pos(P, 2, 5) != 5 * 5 + 2) ++bad;
    }
    std::printf("checked %ld bad %d\n", checked, bad);
    return bad != 0;
}
