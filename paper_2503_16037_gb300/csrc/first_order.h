// Launchers of the first-scattering-order path (single scattering: the
// branch of the method's data flow in Sec. 3 that stops after the direct
// beam).  The radiance then keeps only the first term of the final radiance
// sum of Sec. 2, E_i = e1_i Theta_i(s0 . v), plus the sunlit ground seen
// through the atmosphere; K, s = K^sun e1 and x are not formed.
#pragma once

#include "kern.h"

namespace tk {

// Phase tables (for Theta_i(s0 . v)), extinction and scattering ratios of
// every voxel, and the direct beam T_sun and e1 of every node, in stream
// order on st.  Adds the kernels it launched to *launches.
template <typename T>
void launch_assemble_direct(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                            long long *launches);

// emis[i] = e1_i sum_sp w_sp,i hg_sp(s0 . v) for every atmospheric node i.
template <typename T>
void launch_emission_first(cudaStream_t st, const GridC &g, const FieldP<T> &f, T *emis);

}  // namespace tk
