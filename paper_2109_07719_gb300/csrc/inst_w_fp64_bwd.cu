// Explicit instantiation of the world-aligned adjoint kernels for storage double, D-solves
// double (tape on chip and in global memory; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
BackwardKernel<T> wbackward_kernel(bool onchip) {
  return onchip ? k_wbackward<T, DT, true> : k_wbackward<T, DT, false>;
}
template BackwardKernel<double> wbackward_kernel<double, double>(bool);

}  // namespace host
}  // namespace abasim
