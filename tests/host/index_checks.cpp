// Host checks of the index arithmetic behind the gather tiles, the
// pre-wrapped ray taps, the segment table and the per-direction planes (the
// coupling-selection weights and the edge form's leaving power, read at
// source-relative positions, and the edge form's arrival planes), for a set
// of grid shapes: the
// kernels compute these positions on the device, and every one of them must
// land inside its buffer and on the right node.  Built and run by
// tests/test_host_index_checks.py; prints one line per check and returns the
// number of failing shapes.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "graph.h"

using namespace tg;

namespace {

constexpr int kGroupRows = 128;

// tile gathers of K (transposed = false) or K^T: for every group, row and
// entry, tile layer slot * tl + j must be inside the copied rows and hold the
// haloed position of the entry's source
long check_tiles(const Graph &G, int H, bool transposed) {
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxp = nx + 2 * H, lp = nxp * (ny + 2 * H);
    const int nxy = nx * ny, gpl = (nxy + kGroupRows - 1) / kGroupRows;
    Transposed Tt;
    TileLayout L;
    std::string e;
    if (transposed) {
        transpose_templates(G, H, Tt);
        e = tile_layout(G, Tt, H, L);
    } else {
        e = tile_layout(G, H, L);
    }
    if (!e.empty()) {
        std::printf("  tile layout: %s\n", e.c_str());
        return 1;
    }
    const std::vector<int> &ts = transposed ? Tt.tstart : G.tmpl_start;
    long bad = 0;
    for (int z = 0; z <= nz; ++z)
        for (int q = 0; q < gpl; ++q) {
            const int r0 = q * kGroupRows, r1 = std::min(r0 + kGroupRows - 1, nxy - 1);
            const int y0 = r0 / nx, y1 = r1 / nx, tla = (y1 - y0 + 2 * H + 1) * nxp;
            if (tla > L.tl) ++bad;
            for (int r = r0; r < r0 + kGroupRows; ++r) {
                const int rr = r < nxy ? r : r0;  // rows past the end read the group's first row
                const int y = rr / nx, x = rr - y * nx;
                const int rl = (y - y0 + H) * nxp + x + H, rp = z * lp + (y + H) * nxp + x + H;
                for (int i = ts[z]; i < ts[z + 1]; ++i) {
                    int src;
                    if (transposed) {
                        src = rp + Tt.flat_h[i];
                    } else {
                        const TSlot &t = G.tmpl[i];
                        const int szl = t.sz >= 0 ? t.sz : nz;
                        src = rp + (szl - z) * lp + t.sdy * nxp + t.sdx;
                    }
                    const int ti = L.ttile[i] + rl, ls = ti / L.tl, j = ti % L.tl;
                    if (ti < 0 || ls >= kTileLayers || j >= tla) {
                        ++bad;
                        continue;
                    }
                    const int lay = L.layers[(size_t)z * kTileLayers + ls];
                    if (lay < 0 || lay * lp + y0 * nxp + j != src) ++bad;
                }
            }
        }
    return bad;
}

// pre-wrapped ray taps (column offsets wrapped into the grid, layer offset
// dz nx ny): every cell of every sun ray and ground-chain ray is a node of
// the atmosphere, and the same node as the incremental wrap gives
long check_rays(const Graph &G, const ViewTables &V) {
    const int nx = G.nx, ny = G.ny;
    const long nxy = (long)nx * ny, n_atm = nxy * G.nz;
    long bad = 0;
    auto cell = [&](const Tap &t, int bx, int by) {
        const int dxm = ((t.dx % nx) + nx) % nx, dym = ((t.dy % ny) + ny) % ny;
        int x = bx + dxm, y = by + dym;
        if (x >= nx) x -= nx;
        if (y >= ny) y -= ny;
        return (long)t.dz * nxy + (long)y * nx + x;
    };
    auto ref = [&](const Tap &t, int bx, int by) {
        const int x = ((bx + t.dx) % nx + nx) % nx, y = ((by + t.dy) % ny + ny) % ny;
        return (long)t.dz * nxy + (long)y * nx + x;
    };
    auto ray = [&](const std::vector<Tap> &taps, int off, int n, int bx, int by) {
        if (off < 0 || off + n > (int)taps.size()) {
            ++bad;
            return;
        }
        for (int t = off; t < off + n; ++t) {
            const long c = cell(taps[t], bx, by);
            if (c < 0 || c >= n_atm || c != ref(taps[t], bx, by)) ++bad;
        }
    };
    for (int z = 0; z <= G.nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int Zs = z < G.nz ? z + 1 : 0;
                ray(V.sun_taps, V.sun_off[Zs], V.sun_n[Zs], x, y);
            }
    for (size_t gd = 0; gd < G.gdirs.size(); ++gd)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) ray(G.taps, G.gtop_off[gd], G.gtop_n[gd], x, y);
    return bad;
}

// segment table: the extinction reads of every (voxel, canonical direction)
// and the stores of each entry with its halo copies stay inside the buffers
long check_segments(const Graph &G, int H) {
    std::vector<EdgeDesc> ed;
    std::vector<int> th, dh;
    if (!edge_descriptors(G, H, ed, th, dh).empty()) return 1;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxp = nx + 2 * H;
    const long lp = (long)nxp * (ny + 2 * H), npad = (long)(nz + 1) * lp;
    const long nc = (long)G.canon_dirs.size();
    long bad = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long p = z * lp + (long)(y + H) * nxp + x + H;
                const long ax = x < H ? nx : (x >= nx - H ? -nx : 0);
                const long ay = y < H ? (long)ny * nxp : (y >= ny - H ? -(long)ny * nxp : 0);
                for (long c = 0; c < nc; ++c) {
                    const int u = G.canon_dirs[c];
                    if (z + G.dirs[u][2] < nz) {
                        const int off = G.lat_off[u], n = G.lat_n[u];
                        if (off < 0 || off + n > (int)th.size()) {
                            ++bad;
                            continue;
                        }
                        for (int t = off; t < off + n; ++t)
                            if (p + th[t] < 0 || p + th[t] >= npad) ++bad;
                    }
                    for (long o : {0L, ax, ay, ax + ay})
                        if (c * npad + p + o < 0 || c * npad + p + o >= nc * npad) ++bad;
                }
            }
    return bad;
}

// per-direction planes: for every slot of every row, the source position
// rp + src lies in the source's layer and decodes to the template's source
// node (or one of its halo copies, which the planes hold too); the plane of
// the slot's direction exists (atmospheric sources: n_dirs planes, ground
// sources: n_gdirs) and the edge form's arrival index fits its planes
long check_planes(const Graph &G, int H) {
    std::vector<EdgeDesc> ed;
    std::vector<int> th, dh;
    if (!edge_descriptors(G, H, ed, th, dh).empty()) return 1;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxp = nx + 2 * H;
    const long lp = (long)nxp * (ny + 2 * H), npad = (long)(nz + 1) * lp;
    const int nd = (int)G.dirs.size(), ngd = (int)G.gdirs.size(), nin = nd + ngd, dmax = std::max(nd, ngd);
    const long nxy = (long)nx * ny, n_nodes = nxy * (nz + 1);
    long bad = 0;
    for (int z = 0; z <= nz; ++z)
        for (long r = 0; r < nxy; ++r) {
            const int y = (int)(r / nx), x = (int)(r - (long)y * nx);
            const long rp = z * lp + (long)(y + H) * nxp + x + H, row = z * nxy + r;
            for (int i = G.tmpl_start[z]; i < G.tmpl_start[z + 1]; ++i) {
                const EdgeDesc &d = ed[i];
                const TSlot &t = G.tmpl[i];
                const bool gsrc = (d.bits >> 11) & 1;
                if (gsrc != (t.sz < 0)) ++bad;
                const int szl = t.sz >= 0 ? t.sz : nz;
                const long j = rp + d.src;
                if (j < szl * lp || j >= (szl + 1) * lp) {
                    ++bad;
                    continue;
                }
                const long in = j - szl * lp;
                const int xx = (int)(in % nxp), yy = (int)(in / nxp);
                const int xs = ((xx - H) % nx + nx) % nx, ys = ((yy - H) % ny + ny) % ny;
                if (xs != ((x + t.sdx) % nx + nx) % nx || ys != ((y + t.sdy) % ny + ny) % ny) ++bad;
                if (d.dir < 0 || d.dir >= (gsrc ? ngd : nd) || (long)d.dir * npad + j >= (long)dmax * npad) ++bad;
                const int din = gsrc ? nd + d.dir : d.dir;
                if (din < 0 || din >= nin || (long)din * n_nodes + row >= (long)nin * n_nodes) ++bad;
            }
        }
    return bad;
}

}  // namespace

int main() {
    struct Shape {
        int nx, ny, nz, R;
        double sza, saa, vza, vaa;
    };
    const Shape shapes[] = {{64, 64, 32, 2, 60, 0, 30, 180}, {21, 19, 9, 2, 50, 20, 25, 200},
                            {13, 11, 7, 1, 20, 20, 55, 200}, {9, 10, 2, 2, 50, 20, 25, 200},
                            {5, 5, 1, 1, 30, 0, 0, 0},        {48, 48, 32, 2, 60, 0, 30, 180},
                            {200, 7, 3, 2, 70, 0, 20, 0},     {16, 16, 8, 2, 75, 40, 45, 10}};
    int failing = 0;
    for (const Shape &s : shapes) {
        Graph G;
        std::string e = build_graph(G, s.nx, s.ny, s.nz, 0.05, 0.05, 0.1, s.R, 2048);
        ViewTables V;
        if (e.empty()) e = build_view(G, V, s.sza, s.saa, s.vza, s.vaa, s.nx, s.ny);
        if (!e.empty()) {
            std::printf("%dx%dx%d R%d: %s\n", s.nx, s.ny, s.nz, s.R, e.c_str());
            ++failing;
            continue;
        }
        const long bt = check_tiles(G, s.R, false), btt = check_tiles(G, s.R, true);
        const long br = check_rays(G, V), bs = check_segments(G, s.R), bp = check_planes(G, s.R);
        std::printf("%dx%dx%d R%d: tiles %ld, K^T tiles %ld, rays %ld, segments %ld, planes %ld bad\n", s.nx, s.ny, s.nz,
                    s.R, bt, btt, br, bs, bp);
        if (bt || btt || br || bs || bp) ++failing;
    }
    return failing;
}
