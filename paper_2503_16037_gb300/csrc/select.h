// Coupling selection: the scattering graph keeps the edges whose coupling
// C (Eq. scatt_coup) exceeds c_min (Sec. 2), and each source re-draws its
// quadrature cells (Eq. F_term_phase, Fibonacci lattice of Sec. 3) among the
// directions it keeps.  The chains of the voxel graph keep their slots; a
// dropped chain gets the weight 0.
//
//   kept(j, u)  = the chain has no receiver, or C(j, n1(j, u)) > c_min
//   q'(j, u)    = share of the lattice whose closest kept direction of j is u
//                 (largest cosine, exact ties to the lowest index); ground
//                 sources: cosine-weighted share of the upper hemisphere
//   W(j, u)     = q'(j, u) c(j, u), with the routing weight
//                 c = C sum_v q'_v / sum_v q'_v C_v over the chains of j that
//                 have a receiver (1 without a receiver, without coupling, or
//                 when that sum is 0); the same for the sun weights q'^sun
//
// The decision C > c_min is taken in FP64 from the scene's fields (species
// sums in FP64) in every precision.
#pragma once

#include "kern.h"

namespace tk {

constexpr int kSelMaxDir = 128;  // atmospheric (and ground) directions a source can have

struct SelP {
    double c_min;
    int M;                           // lattice points
    int n_up;                        // lattice points in the upper hemisphere
    int dmax;                        // planes of the weight tables: max(nd, ngd)
    const unsigned char *rank;       // [M][nd] directions by decreasing cosine to each point; points in cell
                                     // order (cell_start of the graph), inside a cell by their rankings
    const double *lat;               // [M][3] the lattice points in that order
    const float4 *latf;              // [M] the same in FP32 (w = 0)
    const double *glat;              // [n_up][3] the upper-hemisphere points in the order of grank
    const float4 *glatf;             // [n_up] the same in FP32
    const float4 *dirf;              // [nd + ngd] unit directions (atmospheric, then ground) in FP32
    const unsigned char *grank;      // [n_up][ngd] ground directions, upper points in ground-cell order
                                     // (inside a cell by their rankings)
    const int *gcell_start;          // [ngd + 1]
    const double *gz;                // [n_up] cosine weight (z) of each upper point
    const double *gzsum;             // [ngd] cosine weight of each ground cell
    double gztot;                    // cosine weight of the upper hemisphere
    double *hgpt;                    // [S][M] HG toward each lattice point (order of the rankings), followed by
                                     // its compute-type copy, the cell sums [S][nd] and the totals [S] in it
    unsigned long long *musmax_bits; // max over voxels of the FP64 total scattering coefficient
    // the re-partition once per distinct kept set
    ulonglong2 *mask;                // [n_nodes] kept set of each source (bit u: direction u)
    int *rep;                        // [n_nodes] source whose re-partition serves this one (-1: none needed)
    int *table;                      // [ht] open-addressing table of kept sets (source index, -1: free)
    int ht;                          // slots: a power of two, at least twice the sources
    int *rlist;                      // [n_nodes] the representative sources, in the order they claimed their slot
    int *rcount;                     // [2] representatives listed, representatives handed out so far
    int *pcnt;                       // [n_nodes][dmax] point counts after the re-draw (representatives only)
    void *ph;                        // [n_nodes][S][dmax] HG (ground: cosine) sums after the re-draw, compute type
};

// Weights W of every (source, direction) for the current fields and
// geometry: w_iso, w_sun [dmax][npad] haloed (the ground sources' planes in
// the ground layer).  Needs the phase tables of the assembly (cell sums).
template <typename T>
void launch_select(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                   const ViewP &vp, const SelP &sp, T *w_iso, T *w_sun, long long *launches);

// The preselected maximum number of couplings: keys[e] = 1 + the bits of the
// FP64 coupling of chain e ([n_atm][nd], then [n_ground][ngd]; 0: the chain
// has no receiver), and one radix-select pass: the histogram hist[2^11] of
// the digit (key >> shift) & (2^width - 1) over the non-zero keys whose bits
// from hi_shift up equal prefix (hi_shift >= 64: all of them); the digit
// is width <= 11 bits wide.
template <typename T>
void launch_topk_keys(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                      unsigned long long *musmax_bits, unsigned long long *keys, long long *launches);
void launch_topk_hist(cudaStream_t st, const unsigned long long *keys, long long n, int shift, int width,
                      int hi_shift, unsigned long long prefix, unsigned int *hist, int nblocks);
constexpr int kTopkDigitBits = 11;
// The threshold in two steps: the radix select on FP32 keys (1 + the bits of
// the FP32 coupling, relative error of a few 1e-7), then the exact FP64 keys
// of the chains whose FP32 coupling lies within a relative band around the
// FP32 threshold (launch_topk_band lists them and counts the chains above
// it; launch_topk_band_keys forms their keys).  band: chain indices; counts:
// [2] chains listed, chains above hi.
template <typename T>
void launch_topk_keys32(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                        unsigned long long *musmax_bits, unsigned int *keys, long long *launches);
void launch_topk_hist32(cudaStream_t st, const unsigned int *keys, long long n, int shift, int width, int hi_shift,
                        unsigned int prefix, unsigned int *hist, int nblocks);
void launch_topk_band(cudaStream_t st, const unsigned int *keys, long long n, double lo, double hi, int *band,
                      int *counts, int nblocks);
template <typename T>
void launch_topk_band_keys(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                           const unsigned long long *musmax_bits, const int *band, int nb, unsigned long long *keys);

// The edge kernel with the weights read from w_iso / w_sun.
template <typename T>
void launch_assemble_rows_sel(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                              const ViewC &vc, const T *w_iso, const T *w_sun, long long *launches);

// The reverse edge march of the adjoint with the weights read from w_iso /
// w_sun (the adjoint of the assembly that launch_assemble_rows_sel made).
template <typename T>
void launch_asm_adj_sel(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                        const double *x64, const double *lam64, const AdjP<T> &ad, const T *w_iso,
                        const T *w_sun);

}  // namespace tk
