// Explicit instantiation of the batched kernels for storage double, D-solves double
// (all kernels; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel() {
  return k_backward<T, DT, ST>;
}
template BackwardKernel<double> backward_kernel<double, double, ST_GLOBAL>();

template int launch_rollout<double, double>(sim_handle*, const void*, const void*, const void*, int64_t, int,
                                      void*, void*, void*, void*, void*);
template int launch_step_with_tape<double, double>(sim_handle*, const void*, const void*, const void*, void*,
                                             void*, void*, void*);
template int launch_backward<double, double>(sim_handle*, const void*, const void*, int64_t, int, const void*,
                                       const void*, const void*, void*, void*, void*, void*, void*, void*);
template int launch_jvp<double>(sim_handle*, const void*, const void*, const void*, const void*, const void*,
                            const void*, void*, void*, void*, void*, void*, void*);
template int launch_set_masses<double>(sim_handle*, const void*, void*);

}  // namespace host
}  // namespace abasim
