// Explicit instantiation of the adjoint kernel for storage float, D-solves double,
// tape and model constants on chip (the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel() {
  return k_backward<T, DT, ST>;
}
template BackwardKernel<float> backward_kernel<float, double, ST_SMEM>();

}  // namespace host
}  // namespace abasim
