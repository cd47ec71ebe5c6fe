// Internal interface between the host side of the C ABI (abasim.cu) and the
// kernel instantiation units (inst_*.cu): the handle and the launch functions,
// explicitly instantiated per precision and direction.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/abasim.h"
#include "aba_step.cuh"

namespace abasim {
namespace host {
constexpr int kDefaultBlock = 32;
}  // namespace host
}  // namespace abasim

struct sim_handle {
  int B = 0, Bpad = 0, maxL = 0, nq_max = 0, nv_max = 0, L_total = 0;
  int precision = SIM_FP64, integrator = SIM_SEMI_IMPLICIT_EULER;
  int block = abasim::host::kDefaultBlock;
  int device = 0;
  double dt = 0, g[3] = {0, 0, 0};
  size_t scalar = 8;
  void* prm = nullptr;       // [maxL][NPRM][B] scalar
  int* meta = nullptr;       // [maxL][B]
  int* nl = nullptr;         // [B]
  int* nqv = nullptr;        // [B]  nq | nv << 16
  void* tape = nullptr;      // [maxL][NTAPE][B] scalar
  void* adj = nullptr;       // [maxL][NADJ][B] scalar
  void* wtape2 = nullptr;    // [maxL][NWT][B] scalar: the pipelined world-aligned adjoint's second tape
  void* wstk = nullptr;      // [2][wdepth][WSW][B] scalar: the world-aligned passes' stacks of parent values
  int wdepth = 0;            // entries a system's stack holds at most (depth-first nesting of its branchings)
  void* gm_acc = nullptr;    // [maxL][B] scalar
  int* link_slot = nullptr;  // [L_total] -> l * B + slot
  int* status = nullptr;     // [B] by system
  int* sys_of_slot = nullptr;  // [B]
  unsigned* counter = nullptr;  // work-unit ticket of persistent launches
  void* ctape = nullptr;     // [maxL][NCT][B] scalar, models with contact spheres only
  void* csys = nullptr;      // [NCS][B] scalar, models with contact spheres only
  double friction = 0.8, erp = 0.2;
  int pgs_iterations = 20;
  int schedule = SIM_SCHED_GRID;
  int tape_space = SIM_TAPE_AUTO;
  int replay = SIM_REPLAY_SEGMENT;
  int prefetch = 2;          // links ahead the world-aligned global-tape passes prefetch
  int last_storage = 0, last_storage_bwd = 0;
  int sms = 0;
  bool all_chains = false;   // every system a serial chain of revolute joints (the pipelined adjoint)
  bool all_revolute = false; // every joint revolute and no contact spheres or limits (the world-aligned kernels)
  bool state64 = false;      // sim_rollout accumulates the state in FP64 (SIM_FP32_D64 only)
  void* x64 = nullptr;       // [nq_max + nv_max][B] double: that state
  std::vector<int> h_sys_of_slot;
  std::string err;
};

namespace abasim {
namespace host {

int fail(sim_handle* h, int code, const std::string& msg);
int cuda_fail(sim_handle* h, cudaError_t e, const char* what);
inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

template <class T, class DT>
int launch_rollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T_, int k,
                   void* ckpt, void* qT, void* qdT, void* traj, void* stream);
template <class T, class DT>
int launch_backward(sim_handle* h, const void* ckpt, const void* tau, int64_t T_, int k,
                    const void* gqT, const void* gqdT, const void* gtraj, void* gq0, void* gqd0,
                    void* gtau, void* gmass, void* work, void* stream);
// one step with the per-link tape at `tape` (any device address) instead of the handle's
template <class T, class DT>
int launch_step_with_tape(sim_handle* h, const void* q, const void* qd, const void* tau, void* q_out,
                          void* qd_out, void* tape, void* stream);
template <class T>
int launch_jvp(sim_handle* h, const void* q, const void* qd, const void* tau, const void* dq,
               const void* dqd, const void* dtau, void* q_out, void* qd_out, void* dq_out,
               void* dqd_out, void* work, void* stream);
template <class T>
int launch_set_masses(sim_handle* h, const void* mass, void* stream);

}  // namespace host
}  // namespace abasim
