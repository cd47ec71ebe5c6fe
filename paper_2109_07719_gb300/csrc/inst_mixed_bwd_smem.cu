// Explicit instantiation of the adjoint kernels for storage float, D-solves double,
// tape and model constants on chip, and the pipelined two-warp variant (the units
// compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel() {
  return k_backward<T, DT, ST>;
}
template BackwardKernel<float> backward_kernel<float, double, ST_SMEM>();

template <class T, class DT>
BackwardKernel<T> backward_pipe_kernel() {
  return k_backward_pipe<T, DT>;
}
template BackwardKernel<float> backward_pipe_kernel<float, double>();

}  // namespace host
}  // namespace abasim
