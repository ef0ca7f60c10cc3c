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
// with Q_j the species mixture of the HG quadrature by arrival direction,
// c the routing weight normalised with Q_j(w -> .), and Lsun the first-order
// leaving power (e1 times the sun weights of the assembly).  The series of
// Eq. fs_sum is iterated until the relative change of X is below the
// requested tolerance.
#pragma once

#include "kern.h"

namespace tk {

template <typename T>
struct AniP {
    T *Q;          // [S][nin][nd] HG quadrature by arrival direction (rows sum to 1)
    double *Qraw;  // [S][nin][nd] cell sums before normalisation
    T *C;          // [n_nodes][nd] coupling of each chain's first receiver (-1: none)
    T *Lsun;       // [n_nodes][nd] first-order leaving power along each direction
    T *Wg;         // [n_ground][ngd] weights q_lamb c of the ground sources
    T *Lh;         // [nd][npad] leaving power, haloed planes (read at source-relative positions)
    double *acc;   // [2] sum of squared changes and of squares of X
};

// Per assembly: the edge kernel writes the raw deposit fraction P of every
// slot into val (instead of K); then couplings, first-order leaving power,
// ground weights and the quadrature tables.
template <typename T>
void launch_assemble_rows_p(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                            const ViewC &vc, long long *launches);
template <typename T>
void launch_aniso_prep(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AniP<T> &a, long long *launches);

// One term of the series: X -> L (haloed planes) -> Xn = rho T L (Xn zeroed
// here), and the change |Xn - X|^2, |Xn|^2 accumulated into a.acc (zeroed here).
template <typename T>
void launch_aniso_step(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const AniP<T> &a, const T *X, T *Xn, long long *launches);

// x (total scattered power, FP64 haloed, for the ground term of the pixels)
// and the emission toward the instrument from X.
template <typename T>
void launch_aniso_finish(cudaStream_t st, const GridC &g, const FieldP<T> &f, const T *X, double *x64, T *emis,
                         long long *launches);

}  // namespace tk
