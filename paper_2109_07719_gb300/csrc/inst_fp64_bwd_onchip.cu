// Explicit instantiation of the adjoint kernels for storage double, D-solves
// double, with the state and input streams (hybrid) or everything (on chip) in
// shared memory (the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel() {
  return k_backward<T, DT, ST>;
}
template BackwardKernel<double> backward_kernel<double, double, ST_HYBRID>();
template BackwardKernel<double> backward_kernel<double, double, ST_SMEM>();

}  // namespace host
}  // namespace abasim
