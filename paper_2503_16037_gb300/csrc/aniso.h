// Anisotropic multiple scattering: the edge unknowns of Eq. flux_system.
// The flux along every directed edge keeps its arrival direction into the
// next scattering, where the phase function p' of Eq. F_term_phase is
// integrated with the angle measured from that direction.  The edges that
// reach a node along one direction are merged (re-emission depends on the
// arrival direction only), so the unknown is X(i, w): the power scattered at
// node i from light that arrived along w (w: the atmospheric directions,
// then the ground chains' directions, nin = nd + ngd of them).
//
//   L(j, u) = Lsun(j, u) + sum_w X(j, w) Q_j(w -> u) c_j(u | w)    atmospheric j
//   L(c, k) = Lsun(c, k) + (sum_w X(c, w)) q_lamb_k c_k            ground c (Lambertian)
//   X(i, w) = rho_i sum_{slots e of row i arriving along w} P_e L(src_e, dir_e)
//
// with Q_j = sum_sp w_sp(j) Q_sp the species mixture of the HG quadrature by
// arrival direction, c the routing weight of the coupling normalised with
// Q_j(w -> .), and Lsun the first-order leaving power (e1 times the sun
// weights of the assembly).
//
// The series itself runs on G = [A B] (and, on the top layers, its zf-free
// form for the directions without a receiver; on the ground x_t q_lamb c):
// per assembly Cf is folded into the deposit fractions, P' = P Cf(src, dir),
// and the first-order term b = rho T Lsun is formed once, so that a term is
//   X' = b + rho sum_slots P' G(src, dir)
// and the contraction's epilogue only stores G.  The FP64 residual keeps
// the unfolded form L = Lsun + Cf G with the plain P.
//
// The routing weight factors: c_j(u | w) = C(j, u) zf(j, w) with
// zf = sum_u' Q_j(w, u') / sum_u' Q_j(w, u') C(j, u') over the directions u'
// that have a receiver, wherever the routing applies at j (coupling on and
// some receiver with C > 0: Q_j > 0 everywhere, so that decision does not
// depend on w), and c = 1 elsewhere.  With
//   A(j, (w, sp)) = w_sp(j) zf(j, w) X(j, w),   B((w, sp), u) = Q_sp(w -> u)
// every term's leaving power is one dense contraction per node tile,
//   L(j, u) = Lsun(j, u) + Cf(j, u) [A B](j, u),   Cf = C or 1,
// for the directions that have a receiver.  A direction without one (it
// leaves through the top; its light still crosses the source's own cell,
// whose self slot reads L) has c = 1; those L come from a second, small
// contraction over the top layers with A = w_sp X.  The denominators of zf
// are one more contraction, per assembly:
//   sqc(j, w) = [A' B'](j, w),  A'(j, (u, sp)) = w_sp(j) C(j, u),  B'((u, sp), w) = Q_sp(w -> u).
// FP32 scenes run the per-term contraction on the tensor cores (tcgen05,
// TF32 operands split in a high and a low part, three products, FP32
// accumulation in tensor memory: a few 1e-6 relative); the per-assembly
// one, whose zf is part of the operator that the FP64 residual refines
// against, and every contraction of FP64 scenes and of the CUDA-core
// variant, run as register-blocked loops on the CUDA cores.  The transport pass is a gather: each arrival direction of a row is
// summed by one warp over the template's slots of that direction, in a fixed
// order, so every term is deterministic.
//
// The series of Eq. fs_sum is iterated until the relative change of X is at
// most the tolerance; the stopping test runs on the device and the host
// reads it every few terms.  FP32 scenes then refine: the residual
// r = F(X) - X of the fixed point X = F(X) is evaluated with X and every
// sum in double-single (FP32 pairs, about 48 bits), and the FP32 series
// solves e = r + (F(e) - F(0)) for the correction, X += e in pairs.
#pragma once

#include "kern.h"

namespace tk {

// tiles of the dense contractions: 128 nodes (the tensor-core M) by all
// outputs; the K dimension runs in chunks of kAniRows rows of X (or of C)
// times the species
constexpr int kAniTileM = 128;
constexpr int kAniRows = 8;

template <typename T>
struct AniP {
    T *Q;           // [S][nin][nd] HG quadrature by arrival direction (rows sum to 1)
    double *Qraw;   // [S][nin][nd] cell sums before normalisation
    T *SQ;          // [nz][S][nin] sum of Q_sp(w -> u) over the u that have a receiver from layer z
    T *CT;          // [nd][n_atm] coupling of each chain's first receiver (0: none)
    T *on;          // [n_atm] 1 where the routing applies, else 0
    T *zf;          // [nin][ldz] the routing factor zf (1 where the routing does not apply)
    T *LsT;         // [nd][n_nodes] first-order leaving power (ground nodes: their ngd directions)
    T *Wg;          // [n_ground][ngd] weights q_lamb c of the ground sources
    T *Lh;          // [nd][npad] leaving power, haloed planes (read at source-relative positions)
    T *CfH;         // [nd][npad] routing coupling Cf of every chain (C where the routing applies, else 1;
                    // ground sources 1), haloed planes
    T *Pc;          // per slot (K's value layout) the deposit fraction times its chain's Cf: P Cf(src, dir)
    T *b;           // [nin][ldx] first-order term rho T Lsun (the series' source)
    T *xtg;         // [n_ground] sum over the arrival directions of the current X (ground nodes)
    T *xtb;         // [n_ground] the same for b (the series' first term)
    const int4 *tslot; // per layer template: its slots in order of arrival direction, {t, src, dir, 0}
                       // (t: template-local index, src and dir as in the slot descriptor)
    const int *tseg;   // [nz + 1][nin + 1] start of each arrival direction's run in tslot
    int max_nt;        // slots of the largest layer template
    int ldx;           // row stride of the [nin][.] node arrays (X, Xn, corrections, residual, X in FP64):
                       // n_nodes rounded up to 32, so that every row starts on 128 bytes
    int ldz;           // row stride of zf: n_atm rounded up to 32
    double *part;   // [transport blocks][2] partial sums of the change of a term
    double *acc;    // [3] sum of squared changes, of squares, relative change of the last checked term
    int *ctl;       // [3] converged flag, terms taken when it was set, blocks of the running transport done
    float *Bl;      // tensor-core operand of the leave contraction (FP32 scenes), split high / low
    float2 *Ads;    // FP32 residual: A split in FP32 pairs, [ani_ds_kp][ldz]
    float2 *Atop;   // the same for the top layers' tiles (A without zf), [ani_ds_kp][ani_ds_ldt]
    float *Bds;     // FP32 residual: B padded to [ani_ds_kp][128]
    int mma;        // 1: contractions on the tensor cores (FP32 scenes)
};

// Operand tables in the tensor cores' layout: chunk c of K holds kAniRows
// rows of X (or C) times S species, kc = kAniRows S values per output row;
// per chunk, the high parts then the low parts, each np x kc values in
// 8 x 4 core matrices (row groups of 8 outputs, 4 K values per 16 bytes).
// The tile widths np (the MMA's N) the tensor-core kernel is built for
// (N = nd <= 128); S >= 3 species use the widest.
__host__ __device__ constexpr int ani_leave_np(int N, int S) {
    return S >= 3 ? 128 : N <= 32 ? 32 : N <= 64 ? 64 : N <= 112 ? 112 : 128;
}
__host__ __device__ constexpr int ani_chunks(int rows) { return (rows + kAniRows - 1) / kAniRows; }
// the FP32 residual's contraction: K padded to 16, the top layers' row
// stride (nodes from the first top tile, rounded up to 64)
inline int ani_ds_kp(int nin, int S) { return (nin * S + 15) / 16 * 16; }
inline int ani_ds_ldt(const GridC &g, int jtop) { return (g.n_atm - jtop + 63) / 64 * 64; }
// floats of a packed operand of `rows` K rows, tile width np
inline size_t ani_btab_floats(int rows, int np, int S) {
    return (size_t)ani_chunks(rows) * 2 * np * kAniRows * S;
}

// Per assembly: the edge kernel writes the raw deposit fraction P of every
// slot into val (instead of K); then couplings, first-order leaving power,
// ground weights, the routing factors zf and the folded form; with `tables`
// also the quadrature tables and the tensor-core operand (they depend on the
// HG asymmetries and the graph only).
template <typename T>
void launch_assemble_rows_p(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                            const ViewC &vc, long long *launches);
template <typename T>
void launch_aniso_prep(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AniP<T> &a, bool tables, long long *launches);

// X, Xn and radd below are [nin][ldx].  a.xtg must hold the ground nodes'
// sums of X over the arrival directions (zero for X = 0); the term leaves
// those of Xn there (the residual pass those of r).
// One term of the series, X -> L (haloed planes) -> Xn = radd + rho T L,
// where L carries Lsun when `sun` is set and radd may be null; then the
// change |Xn - X|^2, |Xn|^2 and the stopping test: the first term whose
// relative change is at most tol sets a.ctl = {1, term}; every kernel of a
// later term returns at once.  a.ctl must be zeroed before the first term
// (the transport's last block takes the test and resets its block count).
// A term is two launches: launch_aniso_leave (the contraction and the
// ground's leaving power of X into a.Lh; cudaErrorInvalidValue, nothing
// launched, when the tensor-core kernel's tensor maps cannot be made), then
// launch_aniso_move (the transport and the stopping test).
template <typename T>
cudaError_t launch_aniso_leave(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                               const AniP<T> &a, const T *X, long long *launches);
template <typename T>
void launch_aniso_move(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const AniP<T> &a, const T *X, T *Xn, const T *radd, bool sun, double tol, int term,
                       long long *launches);

// FP32 refinement, in double-single (FP32 pairs hi + lo, about 48 bits: the
// arithmetic of FP64 on the FP32 units).  The residual r = F(X) - X (F with
// Lsun) of X ([nin][ldx] pairs) with every product accumulated in pairs, L
// the haloed planes [nd][npad] of pairs; r is stored rounded to FP32 and
// a.acc gets |r|^2, |X|^2.
void launch_aniso_resid(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                        const ViewC &vc, const AniP<float> &a, const float2 *X, float2 *L, float *r,
                        long long *launches);
// X += e in pairs (init: X = e)
void launch_aniso_update(cudaStream_t st, long long n, const float *e, float2 *X, bool init);
// x (total scattered power, FP64 haloed, for the ground term of the pixels)
// and the emission toward the instrument from X (type X of the unknowns).
template <typename T, typename XT>
void launch_aniso_finish(cudaStream_t st, const GridC &g, const FieldP<T> &f, const XT *X, int ldx, double *x64,
                         T *emis, long long *launches);

// The solution X(i, w) as [nin][n_nodes] FP64 (from FP32 pairs or FP64).
template <typename XT>
void launch_aniso_export(cudaStream_t st, const GridC &g, const XT *X, int ldx, double *out);

// The two contractions alone, for the tests: out(j, n) for the atmospheric
// nodes j of the current tables, n < N ([N][n_atm]); which: 0 leave (X in
// [nin][ldx]), 1 sqc; mma: the tensor-core kernel, else the CUDA-core one.
cudaError_t launch_aniso_contract_test(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                                       const AniP<float> &a, const float *X, float *out, int which, bool mma);

}  // namespace tk
