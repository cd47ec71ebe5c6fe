// Explicit instantiation of the batched kernels for storage float, D-solves float
// (forward kernels; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template int launch_rollout<float, float>(sim_handle*, const void*, const void*, const void*, int64_t, int,
                                      void*, void*, void*, void*, void*);
template int launch_step_with_tape<float, float>(sim_handle*, const void*, const void*, const void*, void*,
                                             void*, void*, void*);
template int launch_jvp<float>(sim_handle*, const void*, const void*, const void*, const void*, const void*,
                            const void*, void*, void*, void*, void*, void*, void*);
template int launch_set_masses<float>(sim_handle*, const void*, void*);

}  // namespace host
}  // namespace abasim
