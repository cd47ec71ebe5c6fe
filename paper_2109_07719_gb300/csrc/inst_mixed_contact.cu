// Explicit instantiation of the kernels of models with contact spheres for
// storage float, D-solves double (global storage; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT>
RolloutKernel<T> rollout_contact_kernel() {
  return k_rollout<T, DT, ST_GLOBAL, true>;
}
template <class T, class DT>
BackwardKernel<T> backward_contact_kernel() {
  return k_backward<T, DT, ST_GLOBAL, true>;
}
template RolloutKernel<float> rollout_contact_kernel<float, double>();
template BackwardKernel<float> backward_contact_kernel<float, double>();

}  // namespace host
}  // namespace abasim
