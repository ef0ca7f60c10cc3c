// Device-facing structures and kernel launchers of libtursca_gb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tk {

constexpr int MAX_SPECIES = 4;

// One translation-invariant slot class (see graph.h SlotClass), packed.
struct __align__(16) DClass {
    int16_t kind, dir, hgdir, k;
    int16_t bkind, up_idx, gdir, c_one;
    int32_t pre_off, seg_off, hit_off, pad0;
    int16_t pre_n, seg_n, hit_n, n1_ground;
    int16_t n1_dx, n1_dy, n1_dz, pad1;
    double dist1_inv;
    double split;
    int16_t pre_tab, pre_dx, pre_dy, pre_dz;  // segment table lookups (tab < 0: taps)
    int16_t seg_tab, seg_dx, seg_dy, seg_dz;
    float dist1_inv_f, split_f;               // FP32 copies for the FP32 kernels
    float pad2, pad3;
};


// One row-template entry as the edge kernel uses it: every lookup of the
// slot resolved to one offset from the receiver's haloed position rp (so a
// value needs no index arithmetic beyond an add per lookup).
//   src    source node: rp + src
//   pre    tseg index of the segments before the receiver: pre + rp (-1: none or taps)
//   seg    tseg index of the segment ending at the receiver: seg + rp (-1: taps)
//   n1     first chain member of the source (coupling): rt_h[rp + n1]
//   aux    B_TINF: upward direction index; B_TINFG: tinfg index - rp
//   tbase  tap base cell (the source cell): mu_e_h[rp + tbase + tap_h[k]]
//   bits   kind | bkind << 4 | c_one << 8 | n1_ground << 9 | has_pre << 10 | ground source << 11
//   dir    atmospheric direction (q columns), or the ground direction of a ground source
//   taps   pre_n | seg_n << 8 | hit_n << 16, with the lists at pre_off, seg_off, hit_off
//   q, dinv, split  quadrature weight (q_iso or q_lamb), 1 / distance to n1, ground-hit share
struct __align__(16) ASlot {
    int src, pre, seg, n1;
    int aux, tbase, bits, dir;
    int hgdir, taps, pre_off, seg_off;
    int hit_off;
    float q, dinv, split;
    double qd, dinvd, splitd, pad;
};

// Tap offsets (cell offsets relative to the segment base); lengths are in
// separate float / double arrays.
struct __align__(8) DTap {
    int16_t dx, dy, dz, pad;
};

// A tap of a long ray based at column (bx, by) of layer 0: the cell is
// column (bx + (col & 0xffff), by + (col >> 16)) wrapped into the grid, in
// the layer at node offset zoff (= dz nx ny).  Both column offsets are
// stored already wrapped into [0, nx) x [0, ny), so one conditional
// subtraction per axis finds the cell.
struct __align__(8) RTap {
    int col, zoff;
};

// Grid constants shared by most kernels.
struct GridC {
    int nx, ny, nz, nxy, n_atm, n_ground, n_nodes;
    int S, nd, ngd, nup, R, nc;  // nc: canonical directions (segment table rows)
    int wq;                      // warps per 128-row group in the solver passes (4, 6, 8 or 16)
    int wq_em;                   // warps per group in the emission pass
    int gpl;                     // groups of kGroup rows per layer: ceil(nxy / kGroup)
    int ntmax;                   // largest row template (slots per row of a layer)
    // Haloed layout of the solver's node vectors: layer z (z = nz: the ground)
    // is a (ny + 2H) x (nx + 2H) plane, node (x, y, z) at
    // z * lp + (y + H) * nxp + x + H, and the border of width H repeats the
    // periodic partners, so a gather at a column offset of at most H needs no
    // wrap.  H is the largest |sdx|, |sdy| of the row templates.
    int H, nxp, nyp, lp;
    long long npad;              // (nz + 1) * lp
    int stage;                   // 1: FP32 sweeps stage each group's values in shared memory
    int tl;                      // floats per layer of a group's gather tile (0: passes gather from global memory)
    double hx, hy, hz;
};

// Row templates: every receiver row of layer z (z = nz: the ground) has the
// slots tmpl[tstart[z] .. tstart[z+1]); the value of slot t of row r of the
// layer is val[val_base(voff[z], nt, r) + t * kGroup].  A template entry is
// (class, flat, sdx | sdy << 16, sz): source node = row + flat, corrected by
// +-nx when x + sdx leaves [0, nx) and by +-nx*ny when y + sdy leaves
// [0, ny); sz is the absolute source layer (-1: a ground source).
struct GraphP {
    const int *tstart;        // [nz + 2]
    const int4 *tmpl;         // (class, flat, sdx, sdy)
    const long long *voff;    // [nz + 2]
    const DClass *cls;
    const DTap *taps;
    const float *tap_len_f;
    const double *tap_len_d;
    const int4 *dirs;         // (ux, uy, uz, kmax) per atmospheric direction
    const double *dir_len;    // physical length of u
    const double *q_iso;      // [nd]
    const double *q_lamb;     // [ngd]
    const float *q_iso_f;     // FP32 copies of the per-direction constants
    const float *q_lamb_f;
    const float *dir_len_f;
    const float *gdist1_f;
    const int4 *gmem1;        // first member (dx, dy, dzc) of each ground chain
    const double *gdist1;     // distance from the ground point to the first member
    const int *up_dirs;       // atmospheric index of each upward direction
    const int *top_off, *top_n;    // [nup * R]
    const int *lat_off, *lat_n;    // [nd]
    const int *gtop_off, *gtop_n;  // [ngd]
    const RTap *rtaps;             // every tap of the graph as an RTap (read by the ground chains' rays)
    const int *canon_dirs;         // [nc] atmospheric index of each canonical direction
    const int *up_canon;           // [nup] canonical index of each upward direction
    int *status;                   // scene status word (STATUS_* bits; bounded waits set STATUS_TIMEOUT)
    const int *tflat;              // per template entry: source - receiver in the haloed layout
    const ASlot *aslot;            // per template entry: the edge kernel's lookups
    const int *tap_h;              // per tap: haloed offset from the tap's base cell
    const int *dir_h;              // per atmospheric direction: haloed offset of u
    const int *ttile;              // per template entry: the source's offset in a group's gather tile
    const int *tlay;               // [(nz + 1) * kTileLayers] haloed layer copied into each tile layer (-1: none)
    // Runs of the persistent streamed passes: block b of pass kind k (0: all
    // (nz + 1) * gpl groups, 1: the nz * gpl atmospheric groups) handles the
    // groups [run_g[k][b], run_g[k][b + 1]), whose values are
    // [run_v[k][b], run_v[k][b + 1]); run_n[k] blocks.
    const int *run_g[2];
    const long long *run_v[2];
    int run_n[2];
    // lattice segments of the canonical directions, for the segment-table
    // kernel: per canonical direction (first entry in ctap, tap count, u_z, 0)
    // and the graph tap index of each of its taps
    const int4 *cseg;
    const int *ctap;
    int nctap;                     // total taps of the canonical directions
};

// Per-scene optical fields and assembled quantities (element type T).
template <typename T>
struct FieldP {
    const T *mu_a;   // [n_atm]
    const T *mu_s;   // [S][n_atm]
    T *mu_e;         // [n_atm]
    T *mu_st;        // [n_atm]
    T *tsun;         // [n_nodes]
    T *e1;           // [n_nodes]
    T *tinf;         // [nup][n_atm]
    T *tinfg;        // [ngd][lp] haloed ground layer: optical depth from a ground chain's last member to the TOA
    T *a_iso;        // [npad] haloed: coupling factor zc * sqrt(mu_s) of each source (0: weight 1)
    T *a_sun;        // [npad] haloed
    T *tseg;         // [nc][npad] haloed: optical depth of the lattice segment from a node along a canonical direction
    T *rt;           // [n_atm] sqrt of the total scattering coefficient
    T *wsp;          // [S][n_atm] species fractions of the scattering coefficient
    // haloed copies read by the edge kernel at source-relative positions
    T *rt_h;         // [npad]
    T *wsp_h;        // [S][npad]
    T *mu_e_h;       // [npad]
    // [nz][2 ny][2 nx]: the extinction repeated twice along x and y, so that a
    // long ray's cell (x + dx, y + dy) with x, dx in [0, nx) and y, dy in
    // [0, ny) needs no wrap
    T *mu_x;
    T *e1_h;         // [npad]
    T *q_sun;        // [S][nd]
    T *hgv;          // [S][nd + ngd]
    T *hg0v;         // [S]
    T *val;          // [nnz] slot-major per template
    double *cellsum; // [S][nd] HG sums per Fibonacci cell
    T *s;            // [n_nodes]
    T *gsun;         // [n_atm]
    // [npad][srec_stride(S)] haloed source records of the edge kernel:
    // element 0 is a_iso; element 1 + sp, per species, the species share of
    // the scattering coefficient times the first-order power e1 times the sun
    // coupling factor a_sun, negated when the source's sun coupling weight is
    // 1 (a_sun = 0); ground sources carry e1 times a_iso in element 1
    T *srec;
    unsigned long long *mus_max_bits;  // max of mu_s (bits of a non-negative double)
    int *status;     // device status flags
};

struct ViewC {
    double s0[3], v[3], mu0, f0, albedo;
    double g[MAX_SPECIES];
    int coupling;
};

struct ViewP {
    const DTap *sun_taps;
    const RTap *sun_rt;          // the sun taps as RTaps
    const float *sun_len_f;
    const double *sun_len_d;
    const int *sun_off, *sun_n;  // [nz + 1]
    const DTap *los_taps;
    const float *los_len_f;
    const double *los_len_d;
    const int *los_off, *los_n;
    const int *pix_cx, *pix_cy, *pix_cls;
    const double *lattice;       // [M][3] sorted by cell
    const int *cell_start;       // [nd + 1]
    const double *dirhat;        // [nd + ngd][3]
    int npx, npy;
};

enum { STATUS_BAD_FIELD = 1, STATUS_TIMEOUT = 2 };

// per-direction and per-class constants in the compute type, without
// FP64 -> FP32 conversions in FP32 kernels
template <typename T>
struct Cst;
template <>
struct Cst<float> {
    __device__ static __forceinline__ float q_iso(const GraphP &p, int u) { return p.q_iso_f[u]; }
    __device__ static __forceinline__ float q_lamb(const GraphP &p, int u) { return p.q_lamb_f[u]; }
    __device__ static __forceinline__ float dir_len(const GraphP &p, int u) { return p.dir_len_f[u]; }
    __device__ static __forceinline__ float gdist1(const GraphP &p, int u) { return p.gdist1_f[u]; }
    __device__ static __forceinline__ float dinv(const DClass &c) { return c.dist1_inv_f; }
    __device__ static __forceinline__ float split(const DClass &c) { return c.split_f; }
};
template <>
struct Cst<double> {
    __device__ static __forceinline__ double q_iso(const GraphP &p, int u) { return p.q_iso[u]; }
    __device__ static __forceinline__ double q_lamb(const GraphP &p, int u) { return p.q_lamb[u]; }
    __device__ static __forceinline__ double dir_len(const GraphP &p, int u) { return p.dir_len[u]; }
    __device__ static __forceinline__ double gdist1(const GraphP &p, int u) { return p.gdist1[u]; }
    __device__ static __forceinline__ double dinv(const DClass &c) { return c.dist1_inv; }
    __device__ static __forceinline__ double split(const DClass &c) { return c.split; }
};

// Values: per group of kGroup rows of a layer, slot-major inside the group;
// inside one slot row of 128 values, row i of the group (lane i mod 32, row
// block i / 32) sits at 4 (i mod 32) + i / 32, so the four rows a lane owns
// are one aligned 16-byte (FP32) or 32-byte (FP64) quad.
constexpr int kGroup = 128;
__host__ __device__ __forceinline__ int val_lane_pos(int i) { return ((i & 31) << 2) | (i >> 5); }
// stride of the edge kernel's source records (FieldP::srec): a_iso and S sun factors
__host__ __device__ constexpr int srec_stride(int S) { return S <= 3 ? 4 : 8; }
// most taps the canonical lattice segments may have (segment-table kernel)
constexpr int kSegMaxTaps = 512;
// The segment-table kernel's shared-memory tile: a block of kSegTX x kSegTY
// voxels of one layer holds its columns and rows +- R and its layer and the
// R above (R <= 2).
constexpr int kSegTX = 32, kSegTY = 4;
// The canonical lattice segments as kernel parameters, each padded to
// kSegTapsPer taps (zero lengths): tap k of direction c at tile offset
// off[c][k] with length len[c][k]; uz[c] is the direction's z component.
// n = 0 when a segment has more taps than that (the kernel then reads the
// graph's tap lists instead).
constexpr int kSegTapsPer = 4;
template <typename T>
struct SegTab {
    int n;
    int uz[64];
    int off[64][kSegTapsPer];
    T len[64][kSegTapsPer];
};
// source layers a group's gather tile holds (the receiver layer +- R and the ground)
constexpr int kTileLayers = 6;
// largest gather tile (bytes of shared memory per block)
constexpr int kTileMaxBytes = 48 * 1024;
__host__ __device__ __forceinline__ long long val_base(long long voff_z, int nt, int r) {
    return voff_z + (long long)(r / kGroup) * nt * kGroup + val_lane_pos(r % kGroup);
}

// source node of template slot (sdx, sdy, flat) for the receiver at (x, y)
__host__ __device__ __forceinline__ int tmpl_sdx(int4 t) { return (int)(short)(t.z & 0xffff); }
__host__ __device__ __forceinline__ int tmpl_sdy(int4 t) { return (int)(short)((unsigned)t.z >> 16); }
// haloed position of node (x, y, z)
__host__ __device__ __forceinline__ long long halo_pos(const GridC &g, int x, int y, int z) {
    return (long long)z * g.lp + (long long)(y + g.H) * g.nxp + x + g.H;
}

// store v at node (x, y, z)'s haloed position and at each of its halo copies
template <typename T>
__device__ __forceinline__ void store_halo(T *a, const GridC &g, int x, int y, int z, T v) {
    const long long p = halo_pos(g, x, y, z);
    const int ax = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
    const int ay = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    a[p] = v;
    if (ax) a[p + ax] = v;
    if (ay) {
        a[p + ay] = v;
        if (ax) a[p + ax + ay] = v;
    }
}

__host__ __device__ __forceinline__ int slot_src(const GridC &g, int row, int x, int y, int4 t) {
    int sx = x + tmpl_sdx(t), sy = y + tmpl_sdy(t);
    int j = row + t.y;
    j += sx < 0 ? g.nx : 0;
    j -= sx >= g.nx ? g.nx : 0;
    j += sy < 0 ? g.nxy : 0;
    j -= sy >= g.ny ? g.nxy : 0;
    return j;
}

// ---- assembly (kernels_asm.cu)
// CSR export of the slot-major matrix (row order = template order)
// field preparation, quadrature tables, sun, tau_inf sweeps, coupling normalisers
// st[0]: scene stream; st[1..3]: auxiliary streams; ev: five events (no timing)
template <typename T>
void launch_assemble_pre(cudaStream_t const st[4], cudaEvent_t const ev[5], const GridC &g, const GraphP &gp,
                         const FieldP<T> &f, const ViewC &vc, const ViewP &vp, const SegTab<T> &segtab, bool tables,
                         long long *launches);
// the fused edge march + edge weights over all receiver rows
template <typename T>
void launch_assemble_rows(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                          long long *launches);

template <typename T>
void launch_export_csr(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, int32_t *row_ptr,
                       int32_t *col, T *cval, int16_t *dir, int8_t *k);

// ---- solve (kernels_solve.cu)
// y = b + K x (b may be null); T-valued vectors, T accumulation
template <typename T>
void launch_spmv(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y);
// r = s - x + K x in FP64 (x double); partial sums of r^2 into part[nblk]
template <typename T>
void launch_resid64(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *s, const double *x,
                    double *r, double *part, int nblk);
int resid_blocks(const GridC &g);
// warps per 128-row group that fills the GPU's waves best for this grid
int choose_wq(const GridC &g, bool fp64);
// the same residual with FP32-pair (double-single) arithmetic: x = xh + xl
bool resid_ds_ok(const GridC &g);
// true when a group of 128 rows with ntmax template slots can be staged in shared memory (FP32)
bool stage_fits(int ntmax);
void launch_resid_ds(cudaStream_t st, const GridC &g, const GraphP &gp, const float *val, const float *s,
                     const double *x, const float *xh, const float *xl, double *r, double *part, int nblk);
// x += d and (xh, xl may be null) its double-single split
template <typename T>
void launch_update_x(cudaStream_t st, int n, const T *d, double *x, float *xh, float *xl);
// deterministic reductions over the nodes of haloed vectors (halo copies
// skipped): out[k] = sum_nodes V[k*ldv + p] * y[p], k < ncol
template <typename A, typename B>
void launch_dots(cudaStream_t st, const GridC &g, const A *V, size_t ldv, int ncol, const B *y, double *part,
                 int nblk, double *out);
template <typename T>
void launch_sumsq(cudaStream_t st, const GridC &g, const T *x, double *part, int nblk, double *out);
int dot_blocks(const GridC &g);
// haloed dst <- node-ordered src; node-ordered dst <- haloed src
template <typename T, typename U>
void launch_to_halo(cudaStream_t st, const GridC &g, const T *src, U *dst);
template <typename U>
void launch_from_halo(cudaStream_t st, const GridC &g, const U *src, U *dst);
// finalize block partials part[nblk] (single column) into out[0]
void launch_finalize(cudaStream_t st, const double *part, int nblk, double *out);
// finalize two columns part[2][nblk] into out[0..1]
void launch_finalize2(cudaStream_t st, const double *part, int nblk, double *out);
// vector ops
template <typename T, typename U>
void launch_convert(cudaStream_t st, int n, const T *a, U *b);
template <typename T>
void launch_axpy_to64(cudaStream_t st, int n, const T *d, double *x);  // x += d
template <typename T>
void launch_scale(cudaStream_t st, int n, const T *a, double alpha, T *b);  // b = alpha a
// a += b
template <typename T>
void launch_add(cudaStream_t st, int n, T *a, const T *b);
// start of a Chebyshev refinement in one pass: b = (T) r64, d = 0, p = alpha b
template <typename T>
void launch_cheb_start(cudaStream_t st, int n, const double *r64, double alpha, T *b, T *d, T *p);
template <typename T>
void launch_gmres_update(cudaStream_t st, int n, T *w, const T *V, size_t ldv, int k, const double *h);  // w -= V h
// w -= V h, then the interior sum of w^2 into *out (part: scratch of at least
// max(nblk, n / 256 + 1) doubles)
template <typename T>
void launch_gmres_update_norm(cudaStream_t st, const GridC &g, int n, T *w, const T *V, size_t ldv, int k,
                              const double *h, double *part, int nblk, double *out);
template <typename T>
void launch_combine(cudaStream_t st, int n, T *x, const T *V, size_t ldv, int k, const double *y);  // x += V y
// Neumann sweep y = b + K x that also writes per-block sums of (y - x)^2 to part[sweep_blocks]
template <typename T>
void launch_sweep_pow(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y,
                      double *part, double *x64 = nullptr, float *xh = nullptr, float *xl = nullptr);
int sweep_blocks(const GridC &g);
// Chebyshev step: q = K p; r <- r - p + q; d <- d + p; pn = c1 p + c2 r.
// With x64 set (the last step of a refinement) the step also applies
// x64 += d row by row, with the FP32-pair split into xh, xl when those are set.
template <typename T>
void launch_cheb(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *p, T *r, T *d, T *pn,
                 double c1, double c2, double *x64 = nullptr, float *xh = nullptr, float *xl = nullptr);
template <typename T>
void launch_axpby(cudaStream_t st, int n, double a, const T *x, double b, const T *y, T *out);  // out = a x + b y
template <typename T>
void launch_imk(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, T *y);  // y = x - K x

// ---- adjoint (kernels_adjoint.cu)
// Transposed templates of K (rows = sources), see tg::Transposed
struct TransP {
    const int *tstart;       // [nz + 2]
    const long long *voff;   // [nz + 2]
    const int4 *info;        // per entry: (template-local index in the receiver layer, receiver layer, sdx, sdy)
    const int *flat;         // per entry: receiver - source in the haloed layout
    const int *hgdir;        // per entry: scattering-direction index of the slot
};

// adjoint accumulators (compute type); the gradient is mubar
template <typename T>
struct AdjP {
    T *Ebar;      // [n_atm] dJ/dE
    T *Ebar_h;    // [npad]  the same, haloed
    T *e1bar;     // [n_nodes] dJ/de1 (pixels)
    T *e1bar_h;   // [npad]  dJ/de1 (slots), haloed accumulation
    T *xbar;      // [n_nodes] dJ/dx
    T *mubar;     // [n_atm] dJ/dmu_e = dJ/dmu_a
    T *mubar_h;   // [npad]  tap contributions, haloed accumulation
    T *tsegbar;   // [nc][npad]
    T *tinfbar;   // [nup][n_atm]
    T *tinfgbar;  // [ngd][lp]
};

template <typename T>
void launch_transpose_vals(cudaStream_t st, const GridC &g, const GraphP &gp, const TransP &tp, const T *val,
                           T *valT);
template <typename T>
void launch_pix_adj(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                    const T *emis, const double *x, const T *Lbar, const AdjP<T> &ad);
// x-bar += (theta K)^T E-bar over the transposed templates
template <typename T>
void launch_emis_adj(cudaStream_t st, const GridC &g, const GraphP &gpT, const TransP &tp, const FieldP<T> &f,
                     const T *valT, const AdjP<T> &ad);
template <typename T>
void launch_asm_adj(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                    const double *x64, const double *lam64, const AdjP<T> &ad);
template <typename T>
void launch_tables_adj(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AdjP<T> &ad);

// ---- render (kernels_render.cu)
// xc: the solution x in the compute type
template <typename T>
void launch_emission(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                     const T *xc, T *emis);
template <typename T>
void launch_pixels(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                   const T *emis, const double *x, T *rad, T *refl);

}  // namespace tk
