// Explicit instantiation of the pipelined world-aligned adjoint kernel for storage
// float, D-solves float (tapes on chip and in global memory; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
BackwardKernel<T> wbackward_pipe_kernel(bool onchip) {
  return onchip ? k_wbackward_pipe<T, DT, true> : k_wbackward_pipe<T, DT, false>;
}
template BackwardKernel<float> wbackward_pipe_kernel<float, float>(bool);

}  // namespace host
}  // namespace abasim
