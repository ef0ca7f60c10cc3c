// Host-side construction of the voxel scattering graph (see graph.h).
//
// Paper correspondence (Mikkonen et al., scattering graph method):
//   * coupled node pairs and their directions: the scattering graph G(R, L)
//     of Sec. 2 restricted to a voxel stencil; collinear stencil nodes form a
//     chain that shares one quadrature cell (the cell of Eq. F_term_phase
//     excludes "exactly the same direction");
//   * Fibonacci-lattice quadrature: Sec. 3 (phase-function integration,
//     Gonzalez 2010 lattice), each lattice point assigned to the nearest
//     coupled direction;
//   * path integrals stored as lengths per cell, reusable for any field
//     (Sec. 3, path-integral paragraph): the tap tables below.
#include "graph.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <tuple>

namespace tg {

static int igcd(int a, int b) {
    a = std::abs(a);
    b = std::abs(b);
    while (b != 0) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static inline int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Crossing-merge traversal: every parameter at which the path crosses a cell
// face is collected, the list is sorted, and each piece between consecutive
// distinct crossings is attributed to the cell containing its midpoint.
// Coincident crossings (edges, corners) therefore produce no zero-length
// pieces.  For lattice segments between cell centres all crossings are
// multiples of 1/4 and exact in FP64.
bool trace(const double P[3], const double V[3], double tend, double lphys, int bx, int by, int bz, int nz,
           std::vector<Tap> &out) {
    bool ok = true;
    std::vector<double> ts;
    ts.push_back(0.0);
    ts.push_back(tend);
    for (int a = 0; a < 3; ++a) {
        if (V[a] == 0.0) continue;
        double e = P[a] + V[a] * tend;
        double lo = std::min(P[a], e), hi = std::max(P[a], e);
        for (long b = (long)std::floor(lo); b <= (long)std::ceil(hi); ++b) {
            double t = ((double)b - P[a]) / V[a];
            if (t > 0.0 && t < tend) ts.push_back(t);
        }
    }
    std::sort(ts.begin(), ts.end());
    ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
    for (size_t i = 0; i + 1 < ts.size(); ++i) {
        double t0 = ts[i], t1 = ts[i + 1];
        if (!(t1 > t0)) continue;
        double tm = 0.5 * (t0 + t1);
        int c[3];
        for (int a = 0; a < 3; ++a) c[a] = (int)std::floor(P[a] + V[a] * tm);
        if (c[2] < 0 || c[2] >= nz) {
            if (t1 - t0 > 1e-9 * tend) ok = false;
            continue;
        }
        out.push_back(Tap{c[0] - bx, c[1] - by, c[2] - bz, (t1 - t0) * lphys});
    }
    return ok;
}

static std::array<double, 3> unit_phys(const Graph &G, double vx, double vy, double vz, double *len) {
    double a = vx * G.hx, b = vy * G.hy, c = vz * G.hz;
    double L = std::sqrt(a * a + b * b + c * c);
    if (len) *len = L;
    return {a / L, b / L, c / L};
}

static int add_taps(Graph &G, const std::vector<Tap> &t) {
    int off = (int)G.taps.size();
    G.taps.insert(G.taps.end(), t.begin(), t.end());
    return off;
}

std::string build_graph(Graph &G, int nx, int ny, int nz, double hx, double hy, double hz, int R, int M) {
    if (R < 1 || R > 2) return "stencil_radius must be 1 or 2";
    if (nx < 2 * R + 1 || ny < 2 * R + 1) return "nx and ny must be at least 2 * stencil_radius + 1";
    if (nz < R) return "nz must be at least stencil_radius";
    if (!(hx > 0 && hy > 0 && hz > 0)) return "cell sizes must be positive";
    if (M < 64 || M > (1 << 24)) return "fib_points must be in [64, 2^24]";
    if ((long long)nx * ny * (nz + 1) > 200000000LL) return "grid too large";
    G = Graph();
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.hx = hx;
    G.hy = hy;
    G.hz = hz;
    G.R = R;
    G.M = M;
    G.n_atm = nx * ny * nz;
    G.n_ground = nx * ny;
    G.n_nodes = G.n_atm + G.n_ground;
    bool ok_ = true;

    // ---- atmospheric directions: primitive lattice vectors, |u|_inf <= R
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                if (igcd(igcd(dx, dy), dz) != 1) continue;
                G.dirs.push_back({dx, dy, dz});
                int m = std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz)));
                G.kmax.push_back(R / m);
                double L;
                G.uhat.push_back(unit_phys(G, dx, dy, dz, &L));
                G.len.push_back(L);
                if (dz > 0) {
                    G.up_of_dir.push_back((int)G.up_dirs.size());
                    G.up_dirs.push_back((int)G.dirs.size() - 1);
                } else {
                    G.up_of_dir.push_back(-1);
                }
            }
    const int nd = (int)G.dirs.size();
    {
        auto canonical = [](const std::array<int, 3> &u) {
            return u[2] > 0 || (u[2] == 0 && (u[1] > 0 || (u[1] == 0 && u[0] > 0)));
        };
        for (int u = 0; u < nd; ++u)
            if (canonical(G.dirs[u])) G.canon_dirs.push_back(u);
        G.canon_of_dir.assign(nd, -1);
        for (int u = 0; u < nd; ++u)
            for (int c = 0; c < (int)G.canon_dirs.size(); ++c) {
                const auto &v = G.dirs[G.canon_dirs[c]];
                const auto &w = G.dirs[u];
                if ((v[0] == w[0] && v[1] == w[1] && v[2] == w[2]) || (v[0] == -w[0] && v[1] == -w[1] && v[2] == -w[2]))
                    G.canon_of_dir[u] = c;
            }
    }
    // segment s (1-based) of the chain along u, from p_{s-1} to p_s, as a table
    // entry: canonical direction and its start node relative to the source
    auto seg_entry = [&](int u, int s, int &tab, int &dx, int &dy, int &dz) {
        tab = G.canon_of_dir[u];
        bool canon = G.canon_dirs[tab] == u;
        int b = canon ? s - 1 : s;
        dx = b * G.dirs[u][0];
        dy = b * G.dirs[u][1];
        dz = b * G.dirs[u][2];
    };

    // ---- ground directions: (dx, dy, dzc - 1/2); collinear members share a chain
    {
        std::map<std::tuple<int, int, int>, int> key2g;
        for (int dzc = 1; dzc <= R; ++dzc)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    int a = 2 * dx, b = 2 * dy, c = 2 * dzc - 1;
                    int gg = igcd(igcd(a, b), c);
                    auto key = std::make_tuple(a / gg, b / gg, c / gg);
                    auto it = key2g.find(key);
                    int g;
                    if (it == key2g.end()) {
                        g = (int)G.gdirs.size();
                        key2g[key] = g;
                        GroundDir gd;
                        gd.uhat = unit_phys(G, dx, dy, dzc - 0.5, nullptr);
                        G.gdirs.push_back(gd);
                    } else {
                        g = it->second;
                    }
                    G.gdirs[g].mem.push_back({dx, dy, dzc});
                    G.n_gmembers++;
                }
    }
    const int ngd = (int)G.gdirs.size();

    // ---- Fibonacci lattice and nearest-direction partition
    {
        const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
        const double twopi = 2.0 * 3.14159265358979323846;
        G.lattice.resize(M);
        G.cell.resize(M);
        std::vector<long> cnt(nd, 0);
        std::vector<double> zs(ngd, 0.0);
        double ztot = 0.0;
        for (int m = 0; m < M; ++m) {
            double z = 1.0 - (2.0 * m + 1.0) / M;
            double q = m / phi;
            double lam = twopi * (q - std::floor(q));
            double rr = std::sqrt(1.0 - z * z);
            std::array<double, 3> s = {rr * std::cos(lam), rr * std::sin(lam), z};
            G.lattice[m] = s;
            int best = 0;
            double bc = -2.0;
            for (int u = 0; u < nd; ++u) {
                double c = G.uhat[u][0] * s[0] + G.uhat[u][1] * s[1] + G.uhat[u][2] * s[2];
                if (c > bc) {
                    bc = c;
                    best = u;
                }
            }
            G.cell[m] = best;
            cnt[best]++;
            if (s[2] > 0.0) {
                int gb = 0;
                double gc = -2.0;
                for (int g = 0; g < ngd; ++g) {
                    const auto &h = G.gdirs[g].uhat;
                    double c = h[0] * s[0] + h[1] * s[1] + h[2] * s[2];
                    if (c > gc) {
                        gc = c;
                        gb = g;
                    }
                }
                zs[gb] += s[2];
                ztot += s[2];
            }
        }
        G.q_iso.resize(nd);
        for (int u = 0; u < nd; ++u) G.q_iso[u] = (double)cnt[u] / (double)M;
        G.q_lamb.resize(ngd);
        for (int g = 0; g < ngd; ++g) G.q_lamb[g] = zs[g] / ztot;
        // points grouped by cell (stable), for the per-scene HG sums
        G.cell_start.assign(nd + 1, 0);
        for (int m = 0; m < M; ++m) G.cell_start[G.cell[m] + 1]++;
        for (int u = 0; u < nd; ++u) G.cell_start[u + 1] += G.cell_start[u];
        G.cell_order.resize(M);
        std::vector<int> fill(G.cell_start.begin(), G.cell_start.end() - 1);
        for (int m = 0; m < M; ++m) G.cell_order[fill[G.cell[m]]++] = m;
    }

    // ---- lattice taps (centre to next centre along u), relative to the start cell
    G.lat_off.resize(nd);
    G.lat_n.resize(nd);
    std::vector<std::vector<Tap>> lat(nd);
    for (int u = 0; u < nd; ++u) {
        // translation-invariant template: traced from a virtual layer R of a
        // (2R + 1)-layer slab so that every direction stays inside it
        double P[3] = {0.5, 0.5, R + 0.5};
        double V[3] = {(double)G.dirs[u][0], (double)G.dirs[u][1], (double)G.dirs[u][2]};
        ok_ &= trace(P, V, 1.0, G.len[u], 0, 0, R, 2 * R + 1, lat[u]);
        G.lat_off[u] = add_taps(G, lat[u]);
        G.lat_n[u] = (int)lat[u].size();
    }
    auto shifted = [&](int u, int s, std::vector<Tap> &out) {  // lattice taps of the s-th segment (s >= 0)
        for (const Tap &t : lat[u])
            out.push_back(Tap{t.dx + s * G.dirs[u][0], t.dy + s * G.dirs[u][1], t.dz + s * G.dirs[u][2], t.len});
    };

    // ---- partial taps from a top-layer centre to the TOA, per upward direction
    const int nup = (int)G.up_dirs.size();
    G.top_off.assign(nup * R, 0);
    G.top_n.assign(nup * R, 0);
    for (int ui = 0; ui < nup; ++ui) {
        int u = G.up_dirs[ui];
        for (int o = 0; o < G.dirs[u][2]; ++o) {
            int zt = nz - 1 - o;
            if (zt < 0) continue;
            double P[3] = {0.5, 0.5, zt + 0.5};
            double V[3] = {(double)G.dirs[u][0], (double)G.dirs[u][1], (double)G.dirs[u][2]};
            std::vector<Tap> t;
            ok_ &= trace(P, V, (nz - zt - 0.5) / V[2], G.len[u], 0, 0, zt, nz, t);
            G.top_off[ui * R + o] = add_taps(G, t);
            G.top_n[ui * R + o] = (int)t.size();
        }
    }

    // ---- classes and row templates
    std::map<std::vector<long>, int> cls_key;
    auto get_class = [&](const SlotClass &c, const std::vector<long> &key, const std::vector<Tap> &pre,
                         const std::vector<Tap> &seg, const std::vector<Tap> &hit) -> int {
        auto it = cls_key.find(key);
        if (it != cls_key.end()) return it->second;
        SlotClass cc = c;
        cc.pre_off = add_taps(G, pre);
        cc.pre_n = (int)pre.size();
        cc.seg_off = add_taps(G, seg);
        cc.seg_n = (int)seg.size();
        cc.hit_off = add_taps(G, hit);
        cc.hit_n = (int)hit.size();
        int id = (int)G.classes.size();
        G.classes.push_back(cc);
        cls_key[key] = id;
        return id;
    };
    std::vector<std::vector<TSlot>> rows(nz + 1);  // by receiver layer; nz = ground

    for (int sz = 0; sz < nz; ++sz) {
        for (int u = 0; u < nd; ++u) {
            const int ux = G.dirs[u][0], uy = G.dirs[u][1], uz = G.dirs[u][2];
            int m = 0;
            char cs = 'a';
            for (int k = 1; k <= G.kmax[u]; ++k) {
                int rz = sz + k * uz;
                if (rz >= nz) {
                    cs = 'b';
                    break;
                }
                if (rz < 0) {
                    cs = 'c';
                    break;
                }
                m = k;
            }
            // partial segment from the last chain node to the ground
            std::vector<Tap> hit;
            double thit = 0.0, hxp = 0.0, hyp = 0.0;
            if (cs == 'c') {
                double zc = sz + m * uz + 0.5;
                thit = zc / (double)(-uz);
                double P[3] = {0.5 + m * ux, 0.5 + m * uy, zc};
                double V[3] = {(double)ux, (double)uy, (double)uz};
                ok_ &= trace(P, V, thit, G.len[u], 0, 0, sz, nz, hit);
                hxp = P[0] + thit * ux;
                hyp = P[1] + thit * uy;
            }
            for (int k = 1; k <= m; ++k) {
                bool term = (k == m);
                int bk = B_NONE;
                if (term) {
                    if (cs == 'a')
                        bk = uz > 0 ? B_TINF : B_ALL;
                    else if (cs == 'b')
                        bk = B_TINF;
                    else
                        bk = B_HIT;
                }
                SlotClass c;
                c.kind = SK_CHAIN;
                c.dir = u;
                c.hgdir = u;
                c.k = k;
                c.bkind = bk;
                c.n1_dx = ux;
                c.n1_dy = uy;
                c.n1_dz = uz;
                c.dist1 = G.len[u];
                c.up_idx = G.up_of_dir[u];
                std::vector<Tap> pre, seg, h;
                for (int s = 0; s < k - 1; ++s) shifted(u, s, pre);
                shifted(u, k - 1, seg);
                if (k == 2) seg_entry(u, 1, c.pre_tab, c.pre_dx, c.pre_dy, c.pre_dz);
                seg_entry(u, k, c.seg_tab, c.seg_dx, c.seg_dy, c.seg_dz);
                if (bk == B_HIT) h = hit;
                std::vector<long> key = {SK_CHAIN, u, k, bk, bk == B_HIT ? sz : -1, 0, 0};
                int id = get_class(c, key, pre, seg, h);
                rows[sz + k * uz].push_back(TSlot{id, -k * ux, -k * uy, sz, 0});
            }
            if (m == 0) {
                SlotClass c;
                c.kind = SK_SELF;
                c.dir = u;
                c.hgdir = u;
                c.k = 0;
                c.up_idx = G.up_of_dir[u];
                std::vector<Tap> none, h;
                if (cs == 'b') {
                    c.bkind = B_TINF;
                    c.c_one = 1;
                } else {
                    c.bkind = B_HIT;
                    c.n1_ground = 1;
                    c.dist1 = thit * G.len[u];
                    h = hit;
                }
                std::vector<long> key = {SK_SELF, u, 0, c.bkind, cs == 'c' ? sz : -1, 0, 0};
                int id = get_class(c, key, none, none, h);
                rows[sz].push_back(TSlot{id, 0, 0, sz, 0});
            }
            if (cs == 'c') {
                // ground column(s) containing the hit point; exact edge / corner hits split equally
                std::vector<int> xs, ys;
                if (hxp == std::floor(hxp)) {
                    xs = {(int)hxp - 1, (int)hxp};
                } else {
                    xs = {(int)std::floor(hxp)};
                }
                if (hyp == std::floor(hyp)) {
                    ys = {(int)hyp - 1, (int)hyp};
                } else {
                    ys = {(int)std::floor(hyp)};
                }
                double w = 1.0 / (double)(xs.size() * ys.size());
                std::vector<Tap> pre, none;
                for (int s = 0; s < m; ++s) shifted(u, s, pre);
                for (int cx : xs)
                    for (int cy : ys) {
                        SlotClass c;
                        c.kind = SK_GROUND;
                        c.dir = u;
                        c.hgdir = u;
                        c.k = 7;
                        c.bkind = B_HIT;
                        c.split = w;
                        if (m >= 1) {
                            c.n1_dx = ux;
                            c.n1_dy = uy;
                            c.n1_dz = uz;
                            c.dist1 = G.len[u];
                        } else {
                            c.n1_ground = 1;
                            c.dist1 = thit * G.len[u];
                        }
                        if (m == 1) seg_entry(u, 1, c.pre_tab, c.pre_dx, c.pre_dy, c.pre_dz);
                        std::vector<long> key = {SK_GROUND, u, m, B_HIT, sz, cx, cy};
                        int id = get_class(c, key, pre, none, hit);
                        rows[nz].push_back(TSlot{id, -cx, -cy, sz, 0});
                    }
            }
        }
    }

    // ground sources: chains from the ground point through the member voxels
    G.gtop_off.assign(ngd, 0);
    G.gtop_n.assign(ngd, 0);
    for (int g = 0; g < ngd; ++g) {
        const auto &mem = G.gdirs[g].mem;
        int nm = (int)mem.size();
        std::vector<std::vector<Tap>> segs(nm);
        double Pp[3] = {0.5, 0.5, 0.0};
        for (int k = 0; k < nm; ++k) {
            double Q[3] = {0.5 + mem[k][0], 0.5 + mem[k][1], mem[k][2] - 0.5};
            double V[3] = {Q[0] - Pp[0], Q[1] - Pp[1], Q[2] - Pp[2]};
            double L;
            unit_phys(G, V[0], V[1], V[2], &L);
            ok_ &= trace(Pp, V, 1.0, L, 0, 0, 0, nz, segs[k]);
            Pp[0] = Q[0];
            Pp[1] = Q[1];
            Pp[2] = Q[2];
        }
        {  // terminal member to the TOA along the chain direction
            double V[3] = {(double)mem[0][0], (double)mem[0][1], mem[0][2] - 0.5};
            double L;
            unit_phys(G, V[0], V[1], V[2], &L);
            std::vector<Tap> t;
            ok_ &= trace(Pp, V, ((double)nz - Pp[2]) / V[2], L, 0, 0, 0, nz, t);
            G.gtop_off[g] = add_taps(G, t);
            G.gtop_n[g] = (int)t.size();
        }
        double d1;
        unit_phys(G, mem[0][0], mem[0][1], mem[0][2] - 0.5, &d1);
        for (int k = 1; k <= nm; ++k) {
            SlotClass c;
            c.kind = SK_GCHAIN;
            c.dir = -1;
            c.gdir = g;
            c.hgdir = nd + g;
            c.k = k;
            c.bkind = (k == nm) ? B_TINFG : B_NONE;
            c.n1_dx = mem[0][0];
            c.n1_dy = mem[0][1];
            c.n1_dz = mem[0][2] - 1;  // absolute layer of the first member
            c.dist1 = d1;
            std::vector<Tap> pre, none;
            for (int s = 0; s < k - 1; ++s) pre.insert(pre.end(), segs[s].begin(), segs[s].end());
            std::vector<long> key = {SK_GCHAIN, g, k, c.bkind, -1, 0, 0};
            int id = get_class(c, key, pre, segs[k - 1], none);
            rows[mem[k - 1][2] - 1].push_back(TSlot{id, -mem[k - 1][0], -mem[k - 1][1], -1, 0});
        }
    }

    // ---- templates: fixed order (ground sources last; then by source layer, row, column)
    G.tmpl_start.assign(nz + 2, 0);
    G.tmpl_len.assign(nz + 1, 0);
    G.voff.assign(nz + 2, 0);
    const long long nxy = (long long)nx * ny;
    const long long nxy_pad = (nxy + kGroup - 1) / kGroup * kGroup;
    for (int z = 0; z <= nz; ++z) {
        auto &r = rows[z];
        std::stable_sort(r.begin(), r.end(), [](const TSlot &a, const TSlot &b) {
            bool ga = a.sz < 0, gb = b.sz < 0;
            if (ga != gb) return gb;  // atmospheric sources first
            if (a.sz != b.sz) return a.sz < b.sz;
            if (a.sdy != b.sdy) return a.sdy < b.sdy;
            if (a.sdx != b.sdx) return a.sdx < b.sdx;
            return a.cls < b.cls;
        });
        for (auto &t : r) {
            long long src_base = t.sz >= 0 ? (long long)t.sz * nxy : (long long)G.n_atm;
            t.flat = (int)(src_base - (long long)z * nxy + (long long)t.sdy * nx + t.sdx);
        }
        G.tmpl_len[z] = (int)r.size();
        G.max_row = std::max(G.max_row, (int)r.size());
        G.tmpl_start[z + 1] = G.tmpl_start[z] + (int)r.size();
        G.tmpl.insert(G.tmpl.end(), r.begin(), r.end());
        G.voff[z + 1] = G.voff[z] + (long long)r.size() * nxy_pad;
        G.nnz += (long long)r.size() * nxy;
    }
    G.nnz_edges = G.nnz;
    G.nval = G.voff[nz + 1];
    if (G.nval >= (1LL << 31)) return "graph has more than 2^31 slots";
    if (!ok_) return "internal error: a traced segment left the domain";
    return std::string();
}

void expand_csr(const Graph &G, int32_t *row_ptr, int32_t *col, int16_t *dir, int8_t *k) {
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = nx * ny;
    long long e = 0;
    for (int i = 0; i < G.n_nodes; ++i) {
        int z, x, y;
        if (i < G.n_atm) {
            z = i / nxy;
            y = (i / nx) % ny;
            x = i % nx;
        } else {
            z = nz;
            y = (i - G.n_atm) / nx;
            x = (i - G.n_atm) % nx;
        }
        if (row_ptr) row_ptr[i] = (int32_t)e;
        for (int t = G.tmpl_start[z]; t < G.tmpl_start[z + 1]; ++t, ++e) {
            const TSlot &s = G.tmpl[t];
            int sx = wrapi(x + s.sdx, nx), sy = wrapi(y + s.sdy, ny);
            int src = s.sz >= 0 ? (s.sz * ny + sy) * nx + sx : G.n_atm + sy * nx + sx;
            const SlotClass &c = G.classes[s.cls];
            if (col) col[e] = src;
            if (dir) dir[e] = (int16_t)c.hgdir;
            if (k) k[e] = (int8_t)(c.kind == SK_SELF ? 0 : c.kind == SK_GROUND ? 7 : c.k);
        }
    }
    if (row_ptr) row_ptr[G.n_nodes] = (int32_t)e;
}

std::string build_view(const Graph &G, ViewTables &V, double sza, double saa, double vza, double vaa, int npx,
                       int npy) {
    if (!(sza >= 0.0 && sza < 89.9)) return "sza must be in [0, 89.9)";
    if (!(vza >= 0.0 && vza < 89.9)) return "vza must be in [0, 89.9)";
    if (npx < 1 || npy < 1 || (long long)npx * npy > (1LL << 26)) return "bad detector size";
    const double d2r = 3.14159265358979323846 / 180.0;
    V = ViewTables();
    double ts = sza * d2r, ps = saa * d2r, tv = vza * d2r, pv = vaa * d2r;
    V.s0 = {-std::sin(ts) * std::cos(ps), -std::sin(ts) * std::sin(ps), -std::cos(ts)};
    V.v = {std::sin(tv) * std::cos(pv), std::sin(tv) * std::sin(pv), std::cos(tv)};
    V.mu0 = std::cos(ts);
    const int nz = G.nz;
    bool ok_ = true;
    // sun: from (cx + 1/2, cy + 1/2, Zs) toward the sun up to the TOA
    V.sun_off.resize(nz + 1);
    V.sun_n.resize(nz + 1);
    for (int Zs = 0; Zs <= nz; ++Zs) {
        double P[3] = {0.5, 0.5, (double)Zs};
        double D[3] = {-V.s0[0] / G.hx, -V.s0[1] / G.hy, -V.s0[2] / G.hz};
        double tend = ((double)nz - Zs) * G.hz / -V.s0[2];
        std::vector<Tap> t;
        if (Zs < nz) ok_ &= trace(P, D, tend, 1.0, 0, 0, 0, nz, t);
        V.sun_off[Zs] = (int)V.sun_taps.size();
        V.sun_n[Zs] = (int)t.size();
        V.sun_taps.insert(V.sun_taps.end(), t.begin(), t.end());
    }
    // lines of sight, grouped by the sub-cell position of the pixel's ground point
    std::map<std::pair<double, double>, int> cls;
    V.pix_cx.resize((size_t)npx * npy);
    V.pix_cy.resize((size_t)npx * npy);
    V.pix_cls.resize((size_t)npx * npy);
    const double H = nz * G.hz, len = H / V.v[2];
    for (int b = 0; b < npy; ++b)
        for (int a = 0; a < npx; ++a) {
            double gx = (a + 0.5) * G.nx / (double)npx, gy = (b + 0.5) * G.ny / (double)npy;
            int cx = (int)std::floor(gx), cy = (int)std::floor(gy);
            double fx = gx - cx, fy = gy - cy;
            auto key = std::make_pair(fx, fy);
            auto it = cls.find(key);
            int id;
            if (it == cls.end()) {
                id = (int)V.los_off.size();
                cls[key] = id;
                double P[3] = {fx + len * V.v[0] / G.hx, fy + len * V.v[1] / G.hy, (double)nz};
                double D[3] = {-V.v[0] / G.hx, -V.v[1] / G.hy, -V.v[2] / G.hz};
                std::vector<Tap> t;
                ok_ &= trace(P, D, len, 1.0, 0, 0, 0, nz, t);
                V.los_off.push_back((int)V.los_taps.size());
                V.los_n.push_back((int)t.size());
                V.los_taps.insert(V.los_taps.end(), t.begin(), t.end());
            } else {
                id = it->second;
            }
            size_t p = (size_t)b * npx + a;
            V.pix_cx[p] = wrapi(cx, G.nx);
            V.pix_cy[p] = wrapi(cy, G.ny);
            V.pix_cls[p] = id;
        }
    if (!ok_) return "internal error: a traced ray left the domain";
    return std::string();
}

std::string edge_descriptors(const Graph &G, int H, std::vector<EdgeDesc> &out, std::vector<int> &tap_h,
                             std::vector<int> &dir_h) {
    const int nz = G.nz, nxp = G.nx + 2 * H, lp = nxp * (G.ny + 2 * H);
    const long long npad = (long long)(nz + 1) * lp;
    auto inside = [&](int dx, int dy) { return std::abs(dx) <= H && std::abs(dy) <= H; };
    out.assign(G.tmpl.size(), EdgeDesc());
    for (int z = 0; z <= nz; ++z)
        for (int i = G.tmpl_start[z]; i < G.tmpl_start[z + 1]; ++i) {
            const TSlot &t = G.tmpl[i];
            const SlotClass &c = G.classes[t.cls];
            EdgeDesc &d = out[i];
            d = EdgeDesc();
            const bool gsrc = t.sz < 0;
            const int bz = gsrc ? 0 : t.sz;       // base layer of the source's segments and taps
            const int szl = gsrc ? nz : t.sz;     // layer of the source node
            auto rel = [&](int lz, int dx, int dy) { return (lz - z) * lp + (t.sdy + dy) * nxp + (t.sdx + dx); };
            if (!inside(t.sdx, t.sdy)) return "template offset beyond the halo";
            d.src = rel(szl, 0, 0);
            d.pre = -1;
            d.seg = -1;
            if (c.pre_tab >= 0) {
                if (!inside(t.sdx + c.pre_dx, t.sdy + c.pre_dy)) return "segment lookup beyond the halo";
                d.pre = (int)(c.pre_tab * npad + rel(bz + c.pre_dz, c.pre_dx, c.pre_dy));
            }
            if (c.seg_tab >= 0) {
                if (!inside(t.sdx + c.seg_dx, t.sdy + c.seg_dy)) return "segment lookup beyond the halo";
                d.seg = (int)(c.seg_tab * npad + rel(bz + c.seg_dz, c.seg_dx, c.seg_dy));
            }
            // coupling neighbour: always for ground sources (absolute layer n1_dz),
            // for atmospheric sources unless the coupling is 1 or n1 is the ground
            if (gsrc || (!c.c_one && !c.n1_ground)) {
                if (!inside(t.sdx + c.n1_dx, t.sdy + c.n1_dy)) return "coupling lookup beyond the halo";
                d.n1 = rel(gsrc ? c.n1_dz : bz + c.n1_dz, c.n1_dx, c.n1_dy);
            }
            if (c.bkind == B_TINF) d.aux = std::max(c.up_idx, 0);
            if (c.bkind == B_TINFG) d.aux = std::max(c.gdir, 0) * lp - z * lp + t.sdy * nxp + t.sdx;
            d.tbase = rel(bz, 0, 0);
            for (int q = 0; q < 3; ++q) {
                const int off = q == 0 ? c.pre_off : q == 1 ? c.seg_off : c.hit_off;
                const int n = q == 0 ? c.pre_n : q == 1 ? c.seg_n : c.hit_n;
                for (int k = 0; k < n; ++k)
                    if (!inside(t.sdx + G.taps[off + k].dx, t.sdy + G.taps[off + k].dy)) return "tap beyond the halo";
            }
            if (c.pre_n > 255 || c.seg_n > 255 || c.hit_n > 255) return "tap list too long";
            const int has_pre = (c.pre_tab >= 0 || c.pre_n > 0) ? 1 : 0;
            d.bits = c.kind | (c.bkind << 4) | (c.c_one << 8) | (c.n1_ground << 9) | (has_pre << 10) |
                     ((gsrc ? 1 : 0) << 11);
            d.dir = gsrc ? std::max(c.gdir, 0) : std::max(c.dir, 0);
            d.hgdir = c.hgdir;
            d.taps = c.pre_n | (c.seg_n << 8) | (c.hit_n << 16);
            d.pre_off = c.pre_off;
            d.seg_off = c.seg_off;
            d.hit_off = c.hit_off;
            d.q = gsrc ? G.q_lamb[std::max(c.gdir, 0)] : G.q_iso[std::max(c.dir, 0)];
            d.dinv = c.dist1 > 0 ? 1.0 / c.dist1 : 0.0;
            d.split = c.split;
        }
    tap_h.resize(G.taps.size());
    for (size_t k = 0; k < G.taps.size(); ++k) tap_h[k] = G.taps[k].dz * lp + G.taps[k].dy * nxp + G.taps[k].dx;
    dir_h.resize(G.dirs.size());
    for (size_t u = 0; u < G.dirs.size(); ++u) dir_h[u] = G.dirs[u][2] * lp + G.dirs[u][1] * nxp + G.dirs[u][0];
    return std::string();
}

void transpose_templates(const Graph &G, int H, Transposed &T) {
    const int nz = G.nz, nxp = G.nx + 2 * H, lp = nxp * (G.ny + 2 * H);
    const long long nxy = (long long)G.nx * G.ny, nxy_pad = (nxy + kGroup - 1) / kGroup * kGroup;
    std::vector<std::vector<int>> per(nz + 1);  // template indices grouped by source layer
    for (int z = 0; z <= nz; ++z)
        for (int i = G.tmpl_start[z]; i < G.tmpl_start[z + 1]; ++i) {
            const int szl = G.tmpl[i].sz >= 0 ? G.tmpl[i].sz : nz;
            per[szl].push_back(i);
        }
    T.tstart.assign(nz + 2, 0);
    T.voff.assign(nz + 2, 0);
    T.recv_layer.clear();
    T.tmpl_index.clear();
    T.flat_h.clear();
    T.max_row = 0;
    // receiver layer of a template index
    std::vector<int> layer_of(G.tmpl.size());
    for (int z = 0; z <= nz; ++z)
        for (int i = G.tmpl_start[z]; i < G.tmpl_start[z + 1]; ++i) layer_of[i] = z;
    for (int zs = 0; zs <= nz; ++zs) {
        for (int i : per[zs]) {
            const TSlot &t = G.tmpl[i];
            const int zi = layer_of[i];
            T.recv_layer.push_back(zi);
            T.tmpl_index.push_back(i);
            // receiver - source = -(source - receiver)
            T.flat_h.push_back(-((zs - zi) * lp + t.sdy * nxp + t.sdx));
        }
        const int n = (int)per[zs].size();
        T.tstart[zs + 1] = T.tstart[zs] + n;
        T.voff[zs + 1] = T.voff[zs] + (long long)n * nxy_pad;
        T.max_row = std::max(T.max_row, n);
    }
    T.tstart[nz + 1] = (int)T.recv_layer.size();
}

namespace {
// entry e of row layer z (tstart[z] <= e < tstart[z + 1]) gathers from layer
// lay[e] at column offset (dx[e], dy[e])
std::string tile_layout_of(int nx, int ny, int nz, int H, const std::vector<int> &tstart,
                           const std::vector<int> &lay, const std::vector<int> &dx, const std::vector<int> &dy,
                           TileLayout &L) {
    const int nxp = nx + 2 * H;
    const long long nxy = (long long)nx * ny;
    // rows spanned by a group of kGroup rows: at most ceil((kGroup - 1) / nx) + 1
    int span = 0;
    for (long long r0 = 0; r0 < nxy; r0 += kGroup) {
        const long long r1 = std::min(r0 + kGroup - 1, nxy - 1);
        span = std::max(span, (int)(r1 / nx - r0 / nx + 1));
    }
    L.tl = (span + 2 * H) * nxp;
    L.layers.assign((size_t)(nz + 1) * kTileLayers, -1);
    L.ttile.assign(lay.size(), 0);
    for (int z = 0; z <= nz; ++z) {
        int *ls_of = &L.layers[(size_t)z * kTileLayers];
        int n = 0;
        for (int e = tstart[z]; e < tstart[z + 1]; ++e) {
            if (std::abs(dx[e]) > H || std::abs(dy[e]) > H) return "a gather offset lies beyond the halo";
            int ls = -1;
            for (int k = 0; k < n; ++k)
                if (ls_of[k] == lay[e]) ls = k;
            if (ls < 0) {
                if (n == kTileLayers) return "a layer draws on more source layers than a tile holds";
                ls = n;
                ls_of[n++] = lay[e];
            }
            L.ttile[e] = ls * L.tl + dy[e] * nxp + dx[e];
        }
    }
    return std::string();
}
}  // namespace

std::string tile_layout(const Graph &G, int H, TileLayout &L) {
    const size_t n = G.tmpl.size();
    std::vector<int> lay(n), dx(n), dy(n);
    for (size_t i = 0; i < n; ++i) {
        const TSlot &t = G.tmpl[i];
        lay[i] = t.sz >= 0 ? t.sz : G.nz;
        dx[i] = t.sdx;
        dy[i] = t.sdy;
    }
    return tile_layout_of(G.nx, G.ny, G.nz, H, G.tmpl_start, lay, dx, dy, L);
}

std::string tile_layout(const Graph &G, const Transposed &T, int H, TileLayout &L) {
    const size_t n = T.recv_layer.size();
    std::vector<int> lay(n), dx(n), dy(n);
    for (size_t e = 0; e < n; ++e) {
        const TSlot &t = G.tmpl[T.tmpl_index[e]];
        lay[e] = T.recv_layer[e];
        dx[e] = -t.sdx;
        dy[e] = -t.sdy;
    }
    return tile_layout_of(G.nx, G.ny, G.nz, H, T.tstart, lay, dx, dy, L);
}

}  // namespace tg
