"""Which cells of a Block write whole 32-byte sectors (csrc/sector_fill.h),
compiled with the host compiler and checked against a model of the one-cell
sweep's stores: a fluid cell stores its element, an F_FILL cell stores 0 into
its own, an F_PAD cell with j in the flag's top bits also into element
nx + j.  For random rows of fluid, no-slip and moving-wall cells (FP32 and
16-bit element sizes, widths around the sector size, pads on and off):

- every cell the sweep stores lies in a sector that holds a fluid cell (no
  sector of only solid cells is touched);
- every sector that holds a fluid cell and no padding is written whole
  unless it holds a moving-wall cell (only no-slip cells are filled);
- a row's tail sector (the one with padding) is written whole exactly when,
  besides that, pads are on, k = px - nx <= min(nx, 8) and the last k cells
  are all stored;
- F_FILL marks only no-slip cells, F_PAD only the last k cells, with
  j = nx - 1 - x, and never a padding element at or beyond px.
"""
import os
import shutil
import subprocess

import pytest

from paper_1007_1388_gb300 import build

SRC = r"""
#include "sector_fill.h"
#include <cstdio>
#include <random>
#include <vector>

using namespace lbm;

static long long fails = 0, rows_checked = 0, tails_whole = 0, tails_partial = 0;

static void fail(const char *what, int nx, int elem, int pads, int x)
{
    if (fails < 10) std::printf("FAIL %s nx=%d elem=%d pads=%d x=%d\n", what, nx, elem, pads, x);
    ++fails;
}

int main()
{
    std::mt19937 rng(11);
    for (int elem : {4, 2}) {
        const int per = 32 / elem;
        for (int nx = 1; nx <= 70; ++nx) {
            for (int pads = 0; pads < 2; ++pads) {
                const int px = (nx + per - 1) / per * per, k = px - nx;
                const int ny = 3, nz = 2, py = ny + 2;
                const int pxf = (OXF + nx + 1 + 15) / 16 * 16;
                for (int rep = 0; rep < 40; ++rep) {
                    std::vector<uint8_t> f(size_t(pxf) * py * (nz + 2), F_NOSLIP);
                    const double solid = (rep % 4) * 0.25;  // 0, 0.25, 0.5, 0.75
                    for (int z = 0; z < nz; ++z)
                        for (int y = 0; y < ny; ++y)
                            for (int x = 0; x < nx; ++x) {
                                const double r = std::uniform_real_distribution<double>(0, 1)(rng);
                                uint8_t v = r < solid ? F_NOSLIP : F_FLUID;
                                if (r < solid * 0.1) v = F_MOVING;
                                f[((z + 1) * py + (y + 1)) * pxf + x + OXF] = v;
                            }
                    mark_sector_fills(f.data(), nx, ny, nz, px, py, pxf, elem, pads != 0);
                    for (int z = 0; z < nz; ++z)
                        for (int y = 0; y < ny; ++y) {
                            ++rows_checked;
                            const uint8_t *row = &f[((z + 1) * py + (y + 1)) * pxf + OXF];
                            std::vector<int> written(px, 0);
                            for (int x = 0; x < nx; ++x) {
                                const uint8_t v = row[x];
                                const bool fl = (v & F_KIND) == F_FLUID;
                                if ((v & F_FILL) && (v & F_KIND) != F_NOSLIP) fail("fill on a non-no-slip cell", nx, elem, pads, x);
                                if (fl || (v & F_FILL)) written[x] = 1;
                                if (v & F_PAD) {
                                    const int j = v >> F_PAD_SHIFT;
                                    if (!pads) fail("pad without pads", nx, elem, pads, x);
                                    if (x < nx - k) fail("pad on an early cell", nx, elem, pads, x);
                                    if (j != nx - 1 - x) fail("pad index", nx, elem, pads, x);
                                    if (nx + j >= px) fail("pad beyond the row", nx, elem, pads, x);
                                    else written[nx + j] = 1;
                                }
                            }
                            bool tail_stored = pads && k > 0 && k <= nx && k <= 8;
                            for (int x = nx - k; tail_stored && x < nx; ++x)
                                tail_stored = (row[x] & F_KIND) == F_FLUID || (row[x] & F_FILL);
                            for (int s0 = 0; s0 < px; s0 += per) {
                                int any = 0, all = 1, fluid = 0, moving = 0;
                                for (int e = s0; e < s0 + per; ++e) {
                                    any |= written[e];
                                    all &= written[e];
                                    if (e < nx && (row[e] & F_KIND) == F_FLUID) fluid = 1;
                                    if (e < nx && (row[e] & F_KIND) == F_MOVING) moving = 1;
                                }
                                if (any && !fluid) fail("write into a sector without fluid", nx, elem, pads, s0);
                                const bool is_tail = s0 + per > nx && k > 0;
                                if (!fluid) continue;
                                // only moving-wall cells (not filled) leave a sector partial,
                                // and in a row's tail sector the padding unless it is zeroed
                                const bool expect = !moving && (!is_tail || tail_stored);
                                if (expect != bool(all)) fail(is_tail ? "tail sector" : "sector", nx, elem, pads, s0);
                                if (is_tail) (all ? tails_whole : tails_partial)++;
                            }
                        }
                }
            }
        }
    }
    std::printf("%lld %lld %lld %lld\n", rows_checked, tails_whole, tails_partial, fails);
    return fails != 0;
}
"""


def test_sector_fill_writes_whole_sectors(tmp_path):
    cxx = shutil.which("g++")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "fill.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fill"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(cuda, "include"), "-I" + build.CSRC,
                    "-I" + os.path.join(build.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    rows, whole, partial, fails = (int(v) for v in out.stdout.split()[-4:])
    assert out.returncode == 0 and fails == 0, out.stdout
    # both outcomes of the tail rule occur
    assert rows > 30_000 and whole > 100 and partial > 100
