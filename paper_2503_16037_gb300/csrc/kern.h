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
};

// Tap offsets (cell offsets relative to the segment base); lengths are in
// separate float / double arrays.
struct __align__(8) DTap {
    int16_t dx, dy, dz, pad;
};

// Grid constants shared by most kernels.
struct GridC {
    int nx, ny, nz, nxy, n_atm, n_ground, n_nodes;
    int S, nd, ngd, nup, R;
    double hx, hy, hz;
};

// Pointers of the graph (per shape).
struct GraphP {
    const int32_t *row_ptr;
    const int32_t *col;
    const uint16_t *code;
    const DClass *cls;
    const DTap *taps;
    const float *tap_len_f;
    const double *tap_len_d;
    const int4 *dirs;         // (ux, uy, uz, kmax) per atmospheric direction
    const double *dir_len;    // physical length of u
    const double *q_iso;      // [nd]
    const double *q_lamb;     // [ngd]
    const int4 *gmem1;        // first member (dx, dy, dzc) of each ground chain
    const double *gdist1;     // distance from the ground point to the first member
    const int *up_dirs;       // atmospheric index of each upward direction
    const int *top_off, *top_n;    // [nup * R]
    const int *lat_off, *lat_n;    // [nd]
    const int *gtop_off, *gtop_n;  // [ngd]
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
    T *tinfg;        // [ngd][n_ground]
    T *zc_iso;       // [n_nodes]
    T *zc_sun;       // [n_nodes]
    T *q_sun;        // [S][nd]
    T *hgv;          // [S][nd + ngd]
    T *hg0v;         // [S]
    T *val;          // [nnz]
    T *s;            // [n_nodes]
    T *gsun;         // [n_atm]
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

// ---- assembly (kernels_asm.cu)
void launch_expand(cudaStream_t st, const GridC &g, const int *tmpl_start, const int4 *tmpl, const int *tmpl_len,
                   int32_t *row_ptr, int32_t *col, uint16_t *code);
// field preparation, quadrature tables, sun, tau_inf sweeps, coupling normalisers
template <typename T>
void launch_assemble_pre(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                         const ViewP &vp, long long *launches);
// the fused edge march + edge weights over all receiver rows
template <typename T>
void launch_assemble_rows(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                          long long *launches);

// direction and chain index of every slot (from its class)
void launch_slot_info(cudaStream_t st, long long nnz, const uint16_t *code, const DClass *cls, int16_t *dir,
                      int8_t *k, int nd);

// ---- solve (kernels_solve.cu)
// y = b + K x (b may be null); T-valued vectors, T accumulation
template <typename T>
void launch_spmv(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y);
// r = s - x + K x in FP64 (x double); partial sums of r^2 into part[nblk]
template <typename T>
void launch_resid64(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *s, const double *x,
                    double *r, double *part, int nblk);
int resid_blocks(const GridC &g);
// deterministic reductions: out[k] = sum_i V[k*ldv + i] * y[i], k < ncol
template <typename A, typename B>
void launch_dots(cudaStream_t st, int n, const A *V, size_t ldv, int ncol, const B *y, double *part, int nblk,
                 double *out);
template <typename T>
void launch_sumsq(cudaStream_t st, int n, const T *x, double *part, int nblk, double *out);
int dot_blocks(int n);
// finalize block partials part[nblk] (single column) into out[0]
void launch_finalize(cudaStream_t st, const double *part, int nblk, double *out);
// vector ops
template <typename T, typename U>
void launch_convert(cudaStream_t st, int n, const T *a, U *b);
template <typename T>
void launch_axpy_to64(cudaStream_t st, int n, const T *d, double *x);  // x += d
template <typename T>
void launch_scale(cudaStream_t st, int n, const T *a, double alpha, T *b);  // b = alpha a
template <typename T>
void launch_gmres_update(cudaStream_t st, int n, T *w, const T *V, size_t ldv, int k, const double *h);  // w -= V h
template <typename T>
void launch_combine(cudaStream_t st, int n, T *x, const T *V, size_t ldv, int k, const double *y);  // x += V y
template <typename T>
void launch_axpby(cudaStream_t st, int n, double a, const T *x, double b, const T *y, T *out);  // out = a x + b y
template <typename T>
void launch_imk(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, T *y);  // y = x - K x

// ---- render (kernels_render.cu)
template <typename T>
void launch_emission(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                     const double *x, T *emis);
template <typename T>
void launch_pixels(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                   const T *emis, const double *x, T *rad, T *refl);

}  // namespace tk
