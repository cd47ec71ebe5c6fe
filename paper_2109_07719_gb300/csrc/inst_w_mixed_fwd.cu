// Explicit instantiation of the world-aligned rollout kernels for storage float, D-solves
// double (tape on chip and in global memory; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
RolloutKernel<T> wrollout_kernel(bool onchip) {
  return onchip ? k_wrollout<T, DT, true> : k_wrollout<T, DT, false>;
}
template RolloutKernel<float> wrollout_kernel<float, double>(bool);

}  // namespace host
}  // namespace abasim
