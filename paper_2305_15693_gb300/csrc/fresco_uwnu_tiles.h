// Plan-time tiles of the constraint side of the weights-on-a-grid (UwNU) and type-3 (NUwNU)
// plans: host code only, no CUDA. The constraints' positions are fixed for a plan's life, so the
// host orders them once by the tile of the fine grid that holds their cell (their home tile),
// lists for every tile the constraints whose kernel support meets it, and counts for every tile
// the most supports that cover one of its cells (the spread's fixed-point headroom). Within a
// home tile (2D) and within each list, constraints are dealt round-robin over the shared-memory
// bank of their first cell, so the lanes of a warp meet distinct banks.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace fresco {

// Tiles of the fine grid for the type-1 spread: T[a] cells per axis, at most half the axis (so
// a kernel support, at most half the axis too, meets a tile at one periodic shift only), and
// nt[a] tiles per axis (the last one may be shorter). Tile t = (tz nt[1] + ty) nt[0] + tx.
struct UTiles {
    int T[3];
    int nt[3];
};

// The constraint side's order and lists.
struct UTilePlan {
    std::vector<int> perm;       // [n_k] tile order: slot -> the caller's index
    std::vector<int64_t> hoff;   // [n_tiles + 1] slots of each home tile
    std::vector<int64_t> toff;   // [n_tiles + 1] offsets of the tiles' lists in ent
    std::vector<int> ent;        // [n_ent] constraint slots, tile by tile
    std::vector<int> kcov;       // [n_tiles] the most supports that cover one cell of the tile
    int64_t n_ent = 0;
};

// The spread's tiles: up to 32 x 32 cells in 2D and 16 x 8 x 8 in 3D, at most half of each axis
// (the fine grid is even and at least 2w per axis). nf: cells per axis, 1 beyond dim.
inline UTiles utiles_for(int dim, const int nf[3]) {
    static const int t2[3] = {32, 32, 1}, t3[3] = {16, 8, 8};
    UTiles tl{};
    for (int a = 0; a < 3; ++a) {
        tl.T[a] = a < dim ? std::min(dim == 2 ? t2[a] : t3[a], nf[a] / 2) : 1;
        tl.nt[a] = (nf[a] + tl.T[a] - 1) / tl.T[a];
    }
    return tl;
}

// origin and extent of tile t
inline void utile_box(const UTiles &tl, const int nf[3], int64_t t, int o[3], int len[3]) {
    const int tc[3] = {(int)(t % tl.nt[0]), (int)((t / tl.nt[0]) % tl.nt[1]),
                       (int)(t / ((int64_t)tl.nt[0] * tl.nt[1]))};
    for (int a = 0; a < 3; ++a) {
        o[a] = tc[a] * tl.T[a];
        len[a] = std::min(tl.T[a], nf[a] - o[a]);
    }
}

// First support cell, relative to the constraint's cell, for the position f inside the cell as
// the kernels round it (f in T, then ceil(f - w/2) in T).
template <typename T>
inline int usupport_first(double f, int w) {
    const T ft = (T)f;
    return (int)std::ceil((double)(ft - (T)0.5 * (T)w));
}

// First support cell of a constraint along one axis (its cell, its position f), relative to a
// tile's origin o, at the one periodic shift at which the support can meet the tile (extent len).
template <typename T>
inline int usupport_in_tile(int cell, double f, int w, int o, int len, int nf) {
    int d = cell + usupport_first<T>(f, w) - o;
    if (d >= len) d -= nf;
    else if (d + w <= 0) d += nf;
    return d;
}

// Reorders ids[0, n) by dealing them round-robin over the residues key(id) mod 32, so that
// consecutive ids (the lanes of a warp) have distinct residues wherever the range allows.
template <typename Key>
inline void deal_by_residue(int *ids, int64_t n, Key &&key) {
    if (n < 2) return;
    int bucket[33] = {0};
    std::vector<int> keys((size_t)n), by_key((size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        keys[(size_t)j] = (int)(((key(ids[j]) % 32) + 32) % 32);
        ++bucket[keys[(size_t)j] + 1];
    }
    for (int b = 0; b < 32; ++b) bucket[b + 1] += bucket[b];
    int next[32];
    for (int b = 0; b < 32; ++b) next[b] = bucket[b];
    for (int64_t j = 0; j < n; ++j) by_key[(size_t)next[keys[(size_t)j]]++] = ids[j];
    int64_t e = 0;
    for (int r = 0; e < n; ++r)
        for (int b = 0; b < 32; ++b)
            if (bucket[b] + r < bucket[b + 1]) ids[e++] = by_key[(size_t)(bucket[b] + r)];
}

// Builds the plan's order and lists from the constraints' fine cells (cell, [nk][dim], each in
// [0, nf)) and positions inside them (frac, [nk][dim], in [0, 1), rounded to T by the kernels),
// for width w. Returns false when the lists would hold 2^31 entries or more.
//  - perm: a stable counting sort by home tile; in 2D each home tile's constraints are then dealt
//    over the bank of their first window cell in the interpolation (window rows of len_0 + w
//    cells from the tile's origin - floor(w / 2)).
//  - lists: with the position in [0, 1] after rounding, the support's first cell is cell +
//    ceil(f - w/2), so the support lies in [cell - floor(w/2), cell + w - floor(w/2)]; every tile
//    that range meets (per axis, wrapped) lists the constraint, and the kernel clips the exact
//    support to the tile. Each list is dealt over the bank of its entries' first cells in the
//    tile (the spread's threads step through their supports row by row in lockstep).
//  - kcov: per tile, the most exact supports that cover one of its cells.
template <typename T>
bool build_utile_plan(int dim, const int nf[3], int w, const UTiles &tl, const int *cell,
                      const double *frac, int64_t nk, UTilePlan &out) {
    const int64_t n_tiles = (int64_t)tl.nt[0] * tl.nt[1] * tl.nt[2];
    std::vector<int64_t> cnt((size_t)n_tiles + 1, 0);
    std::vector<int64_t> home((size_t)nk);
    for (int64_t q = 0; q < nk; ++q) {
        int64_t t = 0;
        for (int a = dim - 1; a >= 0; --a) t = t * tl.nt[a] + cell[q * dim + a] / tl.T[a];
        home[(size_t)q] = t;
        ++cnt[(size_t)t + 1];
    }
    for (int64_t t = 0; t < n_tiles; ++t) cnt[(size_t)t + 1] += cnt[(size_t)t];
    out.hoff = cnt;
    out.perm.assign((size_t)nk, 0);
    for (int64_t q = 0; q < nk; ++q) out.perm[(size_t)cnt[(size_t)home[(size_t)q]]++] = (int)q;
    if (dim == 2)
        for (int64_t t = 0; t < n_tiles; ++t) {
            int o[3], len[3];
            utile_box(tl, nf, t, o, len);
            const int wl0 = len[0] + w;
            deal_by_residue(&out.perm[(size_t)out.hoff[(size_t)t]],
                            out.hoff[(size_t)t + 1] - out.hoff[(size_t)t], [&](int q) {
                                const int x0 = cell[(size_t)q * 2] - o[0] + w / 2 +
                                               usupport_first<T>(frac[(size_t)q * 2], w);
                                const int y0 = cell[(size_t)q * 2 + 1] - o[1] + w / 2 +
                                               usupport_first<T>(frac[(size_t)q * 2 + 1], w);
                                return (int64_t)y0 * wl0 + x0;
                            });
        }
    // cells and positions in tile order
    std::vector<int> scell((size_t)(nk * dim));
    std::vector<double> sfrac((size_t)(nk * dim));
    for (int64_t i = 0; i < nk; ++i)
        for (int a = 0; a < dim; ++a) {
            scell[(size_t)(i * dim + a)] = cell[(size_t)out.perm[(size_t)i] * dim + a];
            sfrac[(size_t)(i * dim + a)] = frac[(size_t)out.perm[(size_t)i] * dim + a];
        }
    // calls fn(tile) for every tile that lists slot i
    auto for_tiles = [&](int64_t i, auto &&fn) {
        int ta[3][8], na[3];
        for (int a = 0; a < 3; ++a) {
            na[a] = 0;
            if (a >= dim) {
                ta[a][na[a]++] = 0;
                continue;
            }
            const int c = scell[(size_t)(i * dim + a)];
            for (int k = -(w / 2); k <= w - w / 2; ++k) {
                int x = c + k;
                x = x < 0 ? x + nf[a] : (x >= nf[a] ? x - nf[a] : x);
                const int t = x / tl.T[a];
                bool seen = false;
                for (int j = 0; j < na[a]; ++j) seen |= ta[a][j] == t;
                if (!seen && na[a] < 8) ta[a][na[a]++] = t;
            }
        }
        for (int z = 0; z < na[2]; ++z)
            for (int y = 0; y < na[1]; ++y)
                for (int x = 0; x < na[0]; ++x)
                    fn(((int64_t)ta[2][z] * tl.nt[1] + ta[1][y]) * tl.nt[0] + ta[0][x]);
    };
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = 0; i < nk; ++i) for_tiles(i, [&](int64_t t) { ++cnt[(size_t)t + 1]; });
    for (int64_t t = 0; t < n_tiles; ++t) cnt[(size_t)t + 1] += cnt[(size_t)t];
    out.n_ent = cnt[(size_t)n_tiles];
    if (out.n_ent >= (int64_t)1 << 31) return false;
    out.toff = cnt;
    out.ent.assign((size_t)std::max<int64_t>(out.n_ent, 1), 0);
    for (int64_t i = 0; i < nk; ++i)
        for_tiles(i, [&](int64_t t) { out.ent[(size_t)cnt[(size_t)t]++] = (int)i; });
    out.kcov.assign((size_t)n_tiles, 0);
    std::vector<int> cov;
    for (int64_t t = 0; t < n_tiles; ++t) {
        const int64_t e0 = out.toff[(size_t)t], e1 = out.toff[(size_t)t + 1];
        if (e1 == e0) continue;
        int o[3], len[3];
        utile_box(tl, nf, t, o, len);
        auto start = [&](int64_t i, int a) {
            return usupport_in_tile<T>(scell[(size_t)(i * dim + a)], sfrac[(size_t)(i * dim + a)],
                                       w, o[a], len[a], nf[a]);
        };
        deal_by_residue(&out.ent[(size_t)e0], e1 - e0, [&](int i) {
            int st[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) st[a] = a == 0 ? start(i, a) : std::max(start(i, a), 0);
            return ((int64_t)st[2] * len[1] + st[1]) * len[0] + st[0];
        });
        cov.assign((size_t)len[0] * len[1] * len[2], 0);
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t i = out.ent[(size_t)e];
            int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
            for (int a = 0; a < dim; ++a) {
                const int d = start(i, a);
                lo[a] = std::max(d, 0);
                hi[a] = std::min(d + w, len[a]);
            }
            for (int z = lo[2]; z < hi[2]; ++z)
                for (int y = lo[1]; y < hi[1]; ++y)
                    for (int x = lo[0]; x < hi[0]; ++x) ++cov[((size_t)z * len[1] + y) * len[0] + x];
        }
        out.kcov[(size_t)t] = *std::max_element(cov.begin(), cov.end());
    }
    return true;
}

}  // namespace fresco
