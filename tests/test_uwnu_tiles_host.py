"""CPU check of the plan-time tiles of the weights-on-a-grid / type-3 constraint side
(csrc/fresco_uwnu_tiles.h, host code): the order, the tiles' lists and the cover counts that
fresco_uwnu_plan and fresco_nuwnu_plan build, against the arithmetic the kernels do with them.
The program below restates, in plain loops, the spread's clip of each listed support to its
tile and the 2D interpolation's window, and checks on random and adversarial constraint sets:
- perm is a permutation, and every slot of a home tile's range lies in that tile;
- every cell of every constraint's support is written exactly once over all the tiles' lists,
  inside the tile, at the right cell of the periodic fine grid;
- each tile's cover count equals the most supports that cover one of its cells;
- every window read of the 2D interpolation lies inside the staged window (at most 48 cells a
  side) and is the right cell of the fine grid;
- each list holds every slot at most once."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2305_15693_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <vector>
#include "fresco_uwnu_tiles.h"
using namespace fresco;

static uint64_t s_state = 88172645463325252ULL;
static uint64_t next_u64() { s_state ^= s_state << 13; s_state ^= s_state >> 7; s_state ^= s_state << 17; return s_state; }
static double uni() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }
static int below(int n) { return (int)(next_u64() % (uint64_t)n); }
static int wrap(int x, int n) { return ((x % n) + n) % n; }

// mode 0: uniform; 1: crowded into a few cells; 2: positions at the rounding edges, cells at the seam
template <typename T>
long check(int dim, const int nf_in[3], int w, int nk, int mode, long *cells_checked) {
    int nf[3] = {nf_in[0], nf_in[1], dim == 3 ? nf_in[2] : 1};
    const UTiles tl = utiles_for(dim, nf);
    std::vector<int> cell((size_t)nk * dim);
    std::vector<double> frac((size_t)nk * dim);
    // positions where rounding to T moves ceil(f - w/2) (just above 0 and 1/2, just below 1)
    const double edge[6] = {0.0, 1e-12, 0.5, 0.5 + 1e-9, 1.0 - 1e-9, 1.0 - 1e-15};
    for (int q = 0; q < nk; ++q)
        for (int a = 0; a < dim; ++a) {
            int c = below(nf[a]);
            double f = uni();
            if (mode == 1) c = wrap(3 + below(3), nf[a]);
            if (mode == 2) { f = edge[below(6)]; if (below(4) == 0) c = below(2) ? 0 : nf[a] - 1; }
            cell[(size_t)q * dim + a] = c;
            frac[(size_t)q * dim + a] = f;
        }
    UTilePlan p;
    if (!build_utile_plan<T>(dim, nf, w, tl, cell.data(), frac.data(), nk, p)) return 1000000;
    const int64_t n_tiles = (int64_t)tl.nt[0] * tl.nt[1] * tl.nt[2];
    long bad = 0;
    // permutation and home tiles
    std::vector<int> seen((size_t)nk, 0);
    for (int i = 0; i < nk; ++i) ++seen[(size_t)p.perm[(size_t)i]];
    for (int q = 0; q < nk; ++q) bad += seen[(size_t)q] != 1;
    for (int64_t t = 0; t < n_tiles; ++t)
        for (int64_t i = p.hoff[(size_t)t]; i < p.hoff[(size_t)t + 1]; ++i) {
            const int q = p.perm[(size_t)i];
            int64_t h = 0;
            for (int a = dim - 1; a >= 0; --a) h = h * tl.nt[a] + cell[(size_t)q * dim + a] / tl.T[a];
            bad += h != t;
        }
    // the spread's clip, restated: every support cell exactly once
    int ww[3] = {w, w, w};
    for (int a = dim; a < 3; ++a) ww[a] = 1;
    const size_t per = (size_t)ww[0] * ww[1] * ww[2];
    std::vector<int> hits((size_t)nk * per, 0);
    std::vector<int> in_list((size_t)nk, -1);
    for (int64_t t = 0; t < n_tiles; ++t) {
        int o[3], len[3];
        utile_box(tl, nf, t, o, len);
        std::vector<int> cov((size_t)len[0] * len[1] * len[2], 0);
        for (int64_t e = p.toff[(size_t)t]; e < p.toff[(size_t)t + 1]; ++e) {
            const int i = p.ent[(size_t)e];
            if (in_list[(size_t)i] == (int)t) ++bad;   // listed twice in one tile
            in_list[(size_t)i] = (int)t;
            const int q = p.perm[(size_t)i];
            int lo[3] = {0, 0, 0}, k0[3] = {0, 0, 0}, k1[3] = {1, 1, 1}, c0[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) {
                const double f = frac[(size_t)q * dim + a];
                c0[a] = (int)std::ceil((double)((T)f - (T)0.5 * (T)w));
                int d = cell[(size_t)q * dim + a] + c0[a] - o[a];
                if (d >= len[a]) d -= nf[a];
                else if (d + w <= 0) d += nf[a];
                lo[a] = d;
                k0[a] = d < 0 ? -d : 0;
                k1[a] = w < len[a] - d ? w : len[a] - d;
            }
            for (int kz = k0[2]; kz < k1[2]; ++kz)
                for (int ky = k0[1]; ky < k1[1]; ++ky)
                    for (int kx = k0[0]; kx < k1[0]; ++kx) {
                        const int k[3] = {kx, ky, kz};
                        for (int a = 0; a < 3; ++a) {
                            const int l = lo[a] + k[a];
                            if (l < 0 || l >= len[a]) ++bad;
                            else if (a < dim &&
                                     o[a] + l != wrap(cell[(size_t)q * dim + a] + c0[a] + k[a], nf[a]))
                                ++bad;
                        }
                        ++hits[(size_t)q * per + ((size_t)kz * ww[1] + ky) * ww[0] + kx];
                        ++cov[((size_t)(lo[2] + kz) * len[1] + lo[1] + ky) * len[0] + lo[0] + kx];
                    }
        }
        int m = 0;
        for (int v : cov) m = v > m ? v : m;
        bad += m != p.kcov[(size_t)t];
    }
    for (int v : hits) bad += v != 1;
    *cells_checked += (long)hits.size();
    // the 2D window interpolation, restated
    if (dim == 2)
        for (int64_t t = 0; t < n_tiles; ++t) {
            int o[3], len[3];
            utile_box(tl, nf, t, o, len);
            const int ws[2] = {o[0] - w / 2, o[1] - w / 2}, wl[2] = {len[0] + w, len[1] + w};
            if (wl[0] > 48 || wl[1] > 48) ++bad;
            for (int64_t i = p.hoff[(size_t)t]; i < p.hoff[(size_t)t + 1]; ++i) {
                const int q = p.perm[(size_t)i];
                for (int a = 0; a < 2; ++a) {
                    const double f = frac[(size_t)q * 2 + a];
                    const int c0 = (int)std::ceil((double)((T)f - (T)0.5 * (T)w));
                    const int x0 = cell[(size_t)q * 2 + a] + c0 - ws[a];
                    if (x0 < 0 || x0 + w > wl[a]) ++bad;
                    for (int k = 0; k < w; ++k)
                        bad += wrap(ws[a] + x0 + k, nf[a]) != wrap(cell[(size_t)q * 2 + a] + c0 + k, nf[a]);
                }
            }
        }
    return bad;
}

int main() {
    long bad = 0, cells = 0, cases = 0;
    for (int w = 2; w <= 16; ++w)
        for (int dim = 2; dim <= 3; ++dim)
            for (int mode = 0; mode < 3; ++mode)
                for (int rep = 0; rep < 3; ++rep) {
                    int nf[3];
                    for (int a = 0; a < 3; ++a) {
                        const int lo = 2 * w, hi = dim == 2 ? 160 : 48;
                        nf[a] = 2 * ((lo + below(hi > lo ? hi - lo + 1 : 1)) / 2);
                        if (nf[a] < lo) nf[a] = lo;
                    }
                    if (rep == 0) nf[0] = nf[1] = nf[2] = 2 * w;   // the smallest grids
                    const int nk = dim == 2 ? 400 : 120;
                    bad += (mode + rep) % 2 ? check<float>(dim, nf, w, nk, mode, &cells)
                                            : check<double>(dim, nf, w, nk, mode, &cells);
                    ++cases;
                }
    std::printf("%ld %ld %ld\n", bad, cells, cases);
    return 0;
}
"""


def test_constraint_tiles_cover_every_support_cell_once(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("needs a C++ compiler")
    src = tmp_path / "tiles.cpp"
    exe = tmp_path / "tiles"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    bad, cells, cases = int(out[0]), int(out[1]), int(out[2])
    assert cases == 15 * 2 * 3 * 3
    assert cells > 10_000_000
    assert bad == 0
