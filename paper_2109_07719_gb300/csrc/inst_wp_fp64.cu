// Explicit instantiation of the pipelined world-aligned adjoint kernel for storage
// double, D-solves double (tapes on chip and in global memory; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
BackwardKernel<T> wbackward_pipe_kernel(bool onchip) {
  return onchip ? k_wbackward_pipe<T, DT, true> : k_wbackward_pipe<T, DT, false>;
}
template BackwardKernel<double> wbackward_pipe_kernel<double, double>(bool);

}  // namespace host
}  // namespace abasim
