// Host-side graph description of the voxel scattering graph: direction sets,
// Fibonacci-lattice partition, tap tables of every edge segment, and the
// per-layer row templates from which the CSR structure of K is expanded.
//
// Everything here depends only on the grid (shape, spacing, stencil radius,
// lattice size) or on the illumination / viewing geometry, never on the
// optical fields, so it is built once and cached.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace tg {

constexpr int kGroup = 128;  // rows per storage group of the value array

// Slot kinds: what kind of graph edge a stored entry of K is.
enum SlotKind : int {
    SK_CHAIN = 0,  // atmospheric source j deposits on chain node j + k u
    SK_SELF = 1,   // atmospheric source deposits on itself (chain left the domain before p1)
    SK_GROUND = 2, // atmospheric source's chain hits the ground: deposit on a ground column
    SK_GCHAIN = 3  // ground source deposits on a voxel of its chain
};

// What lies beyond a terminal chain node.
enum BeyondKind : int {
    B_NONE = 0,  // not terminal
    B_ALL = 1,   // terminal, nothing beyond (horizontal or downward, stencil ended)
    B_TINF = 2,  // terminal, upward: optical depth to the TOA from the receiver (table)
    B_HIT = 3,   // terminal, the chain reaches the ground: optical depth to the hit point (taps)
    B_TINFG = 4  // terminal node of a ground chain: optical depth to the TOA (table per ground source)
};

struct Tap {
    int dx, dy, dz;  // cell offset relative to the segment's base cell
    double len;      // physical length (km)
};

struct SlotClass {
    int kind = 0, dir = 0, hgdir = 0, k = 0, bkind = B_NONE;
    int pre_off = 0, pre_n = 0;  // taps of the chain segments before the receiver
    int seg_off = 0, seg_n = 0;  // taps of the segment ending at the receiver
    int hit_off = 0, hit_n = 0;  // taps from the last chain node to the ground hit
    int n1_dx = 0, n1_dy = 0, n1_dz = 0, n1_ground = 0;  // first receiver of the chain
    double dist1 = 0.0;          // distance to the first receiver (km)
    double split = 1.0;          // share of a ground hit that falls on this column
    int c_one = 0;               // direction has no receiver other than the source: coupling 1
    int up_idx = -1;             // upward-direction index for B_TINF
    int gdir = -1;               // ground direction index for ground sources
    // full lattice segments are read from the per-node segment table:
    // table index of the segment direction (-1: use the taps) and the node,
    // relative to the source, from which that canonical direction starts
    int pre_tab = -1, pre_dx = 0, pre_dy = 0, pre_dz = 0;
    int seg_tab = -1, seg_dx = 0, seg_dy = 0, seg_dz = 0;
};

// One entry of a row template: the source of a slot relative to the receiver.
struct TSlot {
    int cls;
    int sdx, sdy;  // source column offset (periodic)
    int sz;        // absolute source layer, -1 for a ground source
    int flat;      // source node - receiver node when no periodic wrap occurs
};

struct GroundDir {
    std::vector<std::array<int, 3>> mem;  // (dx, dy, dzc): voxel (c + dx, c + dy, dzc - 1)
    std::array<double, 3> uhat;
};

struct Graph {
    // grid
    int nx = 0, ny = 0, nz = 0, R = 1, M = 0;
    double hx = 0, hy = 0, hz = 0;
    int n_atm = 0, n_ground = 0, n_nodes = 0;

    // atmospheric directions (order: dz, dy, dx ascending from -R)
    std::vector<std::array<int, 3>> dirs;
    std::vector<int> kmax;
    std::vector<std::array<double, 3>> uhat;
    std::vector<double> len;
    std::vector<int> up_of_dir;  // -1 if not upward
    std::vector<int> up_dirs;    // atmospheric index of each upward direction
    // canonical half of the directions (u_z > 0, or u_z = 0 and (u_y > 0 or
    // u_y = 0 and u_x > 0)): one per pair {u, -u}; segment table rows
    std::vector<int> canon_of_dir;  // index of u or -u in canon_dirs
    std::vector<int> canon_dirs;    // atmospheric index of each canonical direction

    // ground directions (collinear members form one chain)
    std::vector<GroundDir> gdirs;
    int n_gmembers = 0;

    // Fibonacci partition
    std::vector<std::array<double, 3>> lattice;  // M unit vectors
    std::vector<int> cell;                       // atmospheric cell of each lattice point
    std::vector<int> cell_order, cell_start;     // lattice points sorted by cell
    std::vector<double> q_iso, q_lamb;

    // taps and classes
    std::vector<Tap> taps;
    std::vector<SlotClass> classes;

    // tau_inf sweep: partial taps from the centre of a top layer to the TOA,
    // per upward direction and start layer offset o (layer nz - 1 - o)
    std::vector<int> top_off, top_n;  // [n_up * R]
    // lattice taps of each direction (segment from a centre to the next)
    std::vector<int> lat_off, lat_n;  // [n_dirs]
    // ground chains: taps from the terminal member to the TOA, per ground direction
    std::vector<int> gtop_off, gtop_n;

    // row templates: layers 0..nz-1, then the ground (index nz).  Every row of
    // a template has the same slots in the same order.  Values are stored per
    // group of kGroup rows of a layer, slot-major inside the group:
    // val[voff[z] + ((r / kGroup) * nt + t) * kGroup + pos(r % kGroup)], with
    // pos(i) = 4 (i mod 32) + i / 32 (the four rows a lane of a 32-wide warp owns
    // are adjacent) (r = row - z * nxy, nt = template length); layers are padded
    // to whole groups.
    std::vector<int> tmpl_start;  // [nz + 2]
    std::vector<TSlot> tmpl;
    std::vector<int> tmpl_len;    // row length per template
    std::vector<long long> voff;  // [nz + 2] first value of each template
    long long nnz = 0, nnz_edges = 0, nval = 0;  // nval: stored values including group padding
    int max_row = 0;
};

// Build the grid-only part.  Returns an empty string on success, else a message.
std::string build_graph(Graph &G, int nx, int ny, int nz, double hx, double hy, double hz, int R, int M);

// One template entry as the edge kernel reads it: every lookup resolved to an
// offset from the receiver's position in the haloed node layout (layer z of
// (ny + 2H) x (nx + 2H), node (x, y, z) at z lp + (y + H)(nx + 2H) + x + H).
//   src    source node;  pre / seg  segment-table index (table * npad + offset), -1: none
//   n1     first chain member of the source (coupling);  tbase  tap base cell (the source cell)
//   aux    upward direction index (B_TINF), or tinfg plane index - receiver position (B_TINFG)
//   bits   kind | bkind << 4 | c_one << 8 | n1_ground << 9 | has_pre << 10 | ground source << 11
//   dir    atmospheric direction, or the ground direction of a ground source
//   taps   pre_n | seg_n << 8 | hit_n << 16 (lists at pre_off, seg_off, hit_off)
//   q      quadrature weight (q_iso or q_lamb);  dinv  1 / distance to n1;  split  ground-hit share
struct EdgeDesc {
    int src, pre, seg, n1, aux, tbase, bits, dir, hgdir, taps, pre_off, seg_off, hit_off;
    double q, dinv, split;
};

// Edge descriptors of every template entry for halo width H, the haloed
// offset of every tap from its base cell, and of every direction.  Fails
// (non-empty message) if a lookup lies more than H columns from its receiver.
std::string edge_descriptors(const Graph &G, int H, std::vector<EdgeDesc> &out, std::vector<int> &tap_h,
                             std::vector<int> &dir_h);

// Shared-memory tiles of the gathered vector for the row-group passes.  The
// sources of a group of 128 rows of layer z lie in at most kTileLayers
// layers (the receiver's layer +- R and the ground) and in the group's rows
// +- H; the tile holds, for each such layer, the rows y0 - H .. y1 + H of the
// haloed layout (y0, y1: first and last row of the group), each layer at a
// stride of tl floats.  A slot's source is then tile[ttile[t] + rl], with rl
// = (y - y0 + H) (nx + 2H) + x + H the row's position inside one tile layer.
constexpr int kTileLayers = 6;
struct TileLayout {
    std::vector<int> ttile;        // per template entry: layer slot * tl + sdy * (nx + 2H) + sdx
    std::vector<int> layers;       // [(nz + 1) * kTileLayers] haloed source layer of each slot, -1: unused
    int tl = 0;                    // floats per tile layer (the largest group span)
};
// Fails (non-empty message) if a layer's templates draw on more than
// kTileLayers source layers.
std::string tile_layout(const Graph &G, int H, TileLayout &L);

// Templates of K^T: for every source layer zs (zs = nz: the ground), the
// template entries of all receiver layers whose source lies in layer zs, in
// a fixed order (receiver layer, then template index).  Because K is
// invariant under horizontal translation, K^T has the same per-layer form:
// the column of entry e of source node j is the receiver j + flat_h[e]
// (haloed offset), and K^T_je = K_{i, tmpl[e]}.
struct Transposed {
    std::vector<int> tstart;        // [nz + 2]
    std::vector<int> recv_layer;    // receiver layer of each entry
    std::vector<int> tmpl_index;    // index of the entry in G.tmpl
    std::vector<int> flat_h;        // receiver - source in the haloed layout (width H)
    std::vector<long long> voff;    // [nz + 2] values of K^T, groups of kGroup source rows, slot-major
    int max_row = 0;
};
void transpose_templates(const Graph &G, int H, Transposed &T);
// The gather tiles of the K^T passes: row layer zs gathers from the receiver
// layers of its entries, at minus the template's column offset.
std::string tile_layout(const Graph &G, const Transposed &T, int H, TileLayout &L);

// Expand the templates into a CSR structure on the host.
void expand_csr(const Graph &G, int32_t *row_ptr, int32_t *col, int16_t *dir, int8_t *k);

// Illumination / viewing geometry tables.
struct ViewTables {
    // sun: tables per start height Zs = 0..nz (0: ground point, z + 1: top face of layer z)
    std::vector<int> sun_off, sun_n;
    std::vector<Tap> sun_taps;
    // line of sight: per pixel class, taps from the TOA down to the ground point,
    // relative to the pixel's ground column; per pixel (cx, cy, class)
    std::vector<int> los_off, los_n;
    std::vector<Tap> los_taps;
    std::vector<int> pix_cx, pix_cy, pix_cls;
    std::array<double, 3> s0, v;  // sun propagation direction, direction to the instrument
    double mu0 = 1.0;
};

std::string build_view(const Graph &G, ViewTables &V, double sza, double saa, double vza, double vaa, int npx,
                       int npy);

// Straight-path traversal: pieces of P + t V, t in [0, tend], by cell; cells are
// absolute (unwrapped) cell coordinates minus (bx, by, bz).  The path must stay
// within layers [0, nz): a piece outside them is dropped if it is a rounding
// sliver at an end point (length below 1e-9 of the path) and is an error
// otherwise (returns false).
bool trace(const double P[3], const double V[3], double tend, double lphys, int bx, int by, int bz, int nz,
           std::vector<Tap> &out);

}  // namespace tg
