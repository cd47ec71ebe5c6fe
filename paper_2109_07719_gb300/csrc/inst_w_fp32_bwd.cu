// Explicit instantiation of the world-aligned adjoint kernels for storage float, D-solves
// float (tape on chip and in global memory; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
BackwardKernel<T> wbackward_kernel(bool onchip) {
  return onchip ? k_wbackward<T, DT, true> : k_wbackward<T, DT, false>;
}
template BackwardKernel<float> wbackward_kernel<float, float>(bool);

}  // namespace host
}  // namespace abasim
