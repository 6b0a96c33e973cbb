// Host side of the one-cell sweep's whole-sector stores: which cells of a
// Block also store the rest state (F_FILL) or zero a padding element (F_PAD).
//
// A PDF plane row holds px >= nx elements of the storage type and starts on a
// 32-byte boundary, so its 32-byte sectors hold per = 32 / elem consecutive
// cells.  The sweep writes every fluid cell.  A no-slip cell in a sector that
// holds a fluid cell is marked F_FILL: the sweep stores 0 there too (its
// PDFs are never read).  With pads, the last k = px - nx cells of a row are
// marked F_PAD with j = nx - 1 - x in the flag's top bits, and each zeroes
// padding element nx + j, when every one of them is stored (fluid or F_FILL)
// and k <= min(nx, 8).  Sectors that hold no fluid cell are not written at all.
#pragma once

#include <algorithm>
#include <cstdint>

#include "sweep_types.h"

namespace lbm {

// f: the Block's flag array, cell (x, y, z) at ((z+1) py + (y+1)) pxf + x + OXF.
inline void mark_sector_fills(uint8_t *f, int nx, int ny, int nz, int px, int py, int pxf, int elem, bool pads)
{
    const int per = 32 / elem, k = px - nx;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            uint8_t *row = f + ((long long)(z + 1) * py + (y + 1)) * pxf + OXF;
            for (int x0 = 0; x0 < nx; x0 += per) {
                const int x1 = std::min(nx, x0 + per);
                bool fluid = false;
                for (int x = x0; x < x1; ++x) fluid = fluid || (row[x] & F_KIND) == F_FLUID;
                if (!fluid) continue;
                for (int x = x0; x < x1; ++x)
                    if ((row[x] & F_KIND) == F_NOSLIP) row[x] |= F_FILL;
            }
            bool tail = pads && k > 0 && k <= nx && k <= 8;  // j < 8 fits the flag's top bits
            for (int x = nx - k; tail && x < nx; ++x) tail = (row[x] & F_KIND) == F_FLUID || (row[x] & F_FILL);
            if (tail)
                for (int x = nx - k; x < nx; ++x) row[x] |= uint8_t(F_PAD | ((nx - 1 - x) << F_PAD_SHIFT));
        }
}

}  // namespace lbm
