// Explicit instantiation of the adjoint kernel for storage float, D-solves float,
// tape in global memory, and its launcher (the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel() {
  return k_backward<T, DT, ST>;
}
template BackwardKernel<float> backward_kernel<float, float, ST_GLOBAL>();

template int launch_backward<float, float>(sim_handle*, const void*, const void*, int64_t, int, const void*,
                                       const void*, const void*, void*, void*, void*, void*, void*, void*);

}  // namespace host
}  // namespace abasim
