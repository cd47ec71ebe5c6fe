// Explicit instantiation of the batched kernels for storage float, D-solves double
// (adjoint kernels; the units compile in parallel).
#include "kernels.cuh"

namespace abasim {
namespace host {

template int launch_backward<float, double>(sim_handle*, const void*, const void*, int64_t, int, const void*,
                                       const void*, const void*, void*, void*, void*, void*, void*, void*);

}  // namespace host
}  // namespace abasim
