// C-ABI implementation: model validation and packing (host), and the batched
// rollout / adjoint kernels (one thread per system, per-link tape in a
// handle-owned scratch laid out [link][field][system] so that neighbouring
// threads touch neighbouring words).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/abasim.h"
#include "aba_step.cuh"
#include "dual.cuh"

using namespace abasim;

namespace {

constexpr int kMaxLinks = 255;
constexpr int kMaxCoords = 1023;
constexpr int kDefaultBlock = 32;

thread_local std::string g_create_error;

}  // namespace

struct sim_handle {
  int B = 0, Bpad = 0, maxL = 0, nq_max = 0, nv_max = 0, L_total = 0;
  int precision = SIM_FP64, integrator = SIM_SEMI_IMPLICIT_EULER;
  int block = kDefaultBlock;
  int device = 0;
  double dt = 0, g[3] = {0, 0, 0};
  size_t scalar = 8;
  void* prm = nullptr;       // [maxL][NPRM][B] scalar
  int* meta = nullptr;       // [maxL][B]
  int* nl = nullptr;         // [B]
  int* nqv = nullptr;        // [B]  nq | nv << 16
  void* tape = nullptr;      // [maxL][NTAPE][B] scalar
  void* adj = nullptr;       // [maxL][NADJ][B] scalar
  void* gm_acc = nullptr;    // [maxL][B] scalar
  int* link_slot = nullptr;  // [L_total] -> l * B + slot
  int* status = nullptr;     // [B] by system
  int* sys_of_slot = nullptr;  // [B]
  unsigned* counter = nullptr;  // work-unit ticket of persistent launches
  int schedule = SIM_SCHED_GRID;
  int tape_space = SIM_TAPE_AUTO;
  int replay = SIM_REPLAY_SEGMENT;
  int sms = 0;
  std::vector<int> h_sys_of_slot;
  std::string err;
};

namespace {

int fail(sim_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(sim_handle* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T> struct DevModel {
  const T* prm;
  const int* meta;
  const int* nl;
  const int* nqv;
  T* tape;
  T* adj;
  int* status;
  const int* sys_of_slot;
  unsigned* counter;
  long long B;
  int maxL;
  int nq_max, nv_max;
  T dt;
  T g0, g1, g2;
  int integ;
  int persistent;
  int smem;
  int quadratic;
};

template <class T> DevModel<T> dev_model(const sim_handle* h) {
  return DevModel<T>{(const T*)h->prm, h->meta, h->nl, h->nqv, (T*)h->tape, (T*)h->adj, h->status,
                     h->sys_of_slot, h->counter, (long long)h->B, h->maxL, h->nq_max, h->nv_max, (T)h->dt,
                     (T)h->g[0], (T)h->g[1], (T)h->g[2], h->integrator, 0, 0,
                     h->replay == SIM_REPLAY_QUADRATIC};
}

extern __shared__ __align__(16) unsigned char g_smem[];

// Scalars per tile (32 systems) a kernel keeps in dynamic shared memory when it
// runs with on-chip storage: the tape (and, for the adjoint, its accumulators and
// the per-link mass-gradient sums), the tile's model constants and meta words,
// its working state (x for the forward rollout, the state adjoint for the
// backward one) and a double buffer for the per-step input streams (tau, plus the
// checkpointed state for the adjoint) fetched one step ahead.
__host__ __device__ __forceinline__ long long smem_per_tile(int maxL, int nx, int nv, bool bwd) {
  return (long long)maxL * (NTAPE + NPRM + 1 + (bwd ? NADJ + 1 : 0)) + nx + 2LL * (nv + (bwd ? nx : 0));
}

// On-chip regions of one tile, [tile in block] outermost, lane innermost.
template <class T> struct SmemTile {
  T* tape;
  T* adj;
  T* prm;
  int* meta;
  T* state;
  T* gm;
  T* stream;
};

template <class T, bool BWD>
__device__ __forceinline__ SmemTile<T> smem_tile(int maxL, int nx, int nv, int lane) {
  const int tb = threadIdx.x / LANES;
  const long long L = maxL;
  T* base = reinterpret_cast<T*>(g_smem) + (long long)tb * smem_per_tile(maxL, nx, nv, BWD) * LANES + lane;
  SmemTile<T> t;
  t.tape = base;
  base += L * NTAPE * LANES;
  t.adj = base;
  if (BWD) base += L * NADJ * LANES;
  t.prm = base;
  base += L * NPRM * LANES;
  t.meta = reinterpret_cast<int*>(base);  // one scalar slot per int (T is 4 or 8 bytes)
  base += L * LANES;
  t.state = base;
  base += (long long)nx * LANES;
  t.gm = base;
  if (BWD) base += L * LANES;
  t.stream = base;
  return t;
}

// Asynchronous global -> shared copies (cp.async), one element per call.
template <class T> __device__ __forceinline__ void cp_async(T* smem_dst, const T* gsrc) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_newest() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// With SMEM the tile's tape, constants, meta words and working state live in
// shared memory (copied in here); otherwise the tapes are in the handle's global
// scratch and the constants are read from global memory.
template <class T, bool SMEM, bool BWD>
__device__ __forceinline__ Sys<T> sys_of(const DevModel<T>& m, int slot) {
  const long long tile = slot / LANES, lane = slot % LANES;
  const long long L = m.maxL;
  const T* gprm = m.prm + tile * L * NPRM * LANES + lane;
  const int* gmeta = m.meta + tile * L * LANES + lane;
  if (SMEM) {
    const SmemTile<T> st = smem_tile<T, BWD>(m.maxL, m.nq_max + m.nv_max, m.nv_max, (int)lane);
    const int nl = m.nl[slot];
    for (int l = 0; l < nl; ++l) {
      for (int f = 0; f < NPRM; ++f) st.prm[(l * NPRM + f) * LANES] = gprm[(l * NPRM + f) * LANES];
      st.meta[l * LANES * (int)(sizeof(T) / sizeof(int))] = gmeta[l * LANES];
    }
    return Sys<T>{st.prm, st.meta, st.tape, st.adj, nl, (int)(sizeof(T) / sizeof(int))};
  }
  return Sys<T>{gprm, gmeta, m.tape + tile * L * NTAPE * LANES + lane,
                m.adj + tile * L * NADJ * LANES + lane, m.nl[slot], 1};
}

template <class T> __device__ __forceinline__ bool finite_t(T x) { return isfinite(x); }

// ------------------------------------------------------------------ kernels
// Thread i of the launch handles slot i.  Slots hold the systems sorted by link
// count (longest first) so a warp's systems walk the same number of links; the
// model constants and tapes are stored by slot, the caller's arrays by system.

// T steps of one system.  The working state lives in (qT, qdT); checkpoints every
// k steps; optional full trajectory.
template <class T, class DT, bool SMEM>
__device__ __forceinline__ void rollout_one(const DevModel<T>& m, int slot, const T* __restrict__ q0,
                                            const T* __restrict__ qd0, const T* __restrict__ tau,
                                            long long Tn, int k, T* ckpt, T* qT, T* qdT, T* traj) {
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const V3<T> g{m.g0, m.g1, m.g2};
  Sys<T> s = sys_of<T, SMEM, false>(m, slot);
  Col<T> q{qT + b, B}, qd{qdT + b, B};
  T* sbuf = nullptr;  // [2][nvm][LANES] double buffer for tau
  if (SMEM) {  // the working state on chip; written to (qT, qdT) at the end
    const SmemTile<T> st = smem_tile<T, false>(m.maxL, NX, nvm, slot % LANES);
    q = Col<T>{st.state, LANES};
    qd = Col<T>{st.state + nqm * LANES, LANES};
    sbuf = st.stream;
    if (Tn > 0)
      for (int d = 0; d < nvm; ++d) cp_async(sbuf + d * LANES, tau + (long long)d * B + b);
    cp_commit();
  }
  for (int d = 0; d < nqm; ++d) q[d] = q0[d * B + b];
  for (int d = 0; d < nvm; ++d) qd[d] = qd0[d * B + b];
  if (traj) {
    for (int d = 0; d < nqm; ++d) traj[d * B + b] = q[d];
    for (int d = 0; d < nvm; ++d) traj[(nqm + d) * B + b] = qd[d];
  }
  for (long long t = 0; t < Tn; ++t) {
    if (ckpt && t % k == 0) {
      T* c = ckpt + (t / k) * NX * B + b;
      for (int d = 0; d < nqm; ++d) c[d * B] = q[d];
      for (int d = 0; d < nvm; ++d) c[(nqm + d) * B] = qd[d];
    }
    Col<const T> tau_t{tau + t * nvm * B + b, B};
    if (SMEM) {  // fetch tau^{t+1} while step t runs
      if (t + 1 < Tn) {
        T* nb = sbuf + ((t + 1) & 1) * nvm * LANES;
        for (int d = 0; d < nvm; ++d) cp_async(nb + d * LANES, tau + ((t + 1) * nvm + d) * B + b);
      }
      cp_commit();
      cp_wait_all_but_newest();
      tau_t = Col<const T>{sbuf + (t & 1) * nvm * LANES, LANES};
    }
    aba_forward<T, DT, false>(s, Col<const T>{q.p, q.B}, Col<const T>{qd.p, qd.B}, tau_t, g);
    integrate<T>(s, q, qd, m.dt, m.integ);
    if (traj) {
      T* c = traj + (t + 1) * NX * B + b;
      for (int d = 0; d < nqm; ++d) c[d * B] = q[d];
      for (int d = 0; d < nvm; ++d) c[(nqm + d) * B] = qd[d];
    }
  }
  if (SMEM) cp_wait_all();
  bool ok = true;
  for (int d = 0; d < nqm; ++d) ok &= finite_t(q[d]);
  for (int d = 0; d < nvm; ++d) ok &= finite_t(qd[d]);
  if (!ok) m.status[b] |= 1;
  if (SMEM) {
    for (int d = 0; d < nqm; ++d) qT[d * B + b] = q[d];
    for (int d = 0; d < nvm; ++d) qdT[d * B + b] = qd[d];
  }
}

// Adjoint rollout of one system.  (gq0, gqd0) carry the running state adjoint
// R^t = xbar^t.
template <class T, class DT, bool SMEM>
__device__ __forceinline__ void backward_one(const DevModel<T>& m, int slot, const T* __restrict__ ckpt,
                                             const T* __restrict__ tau, long long Tn, int k,
                                             const T* __restrict__ gqT, const T* __restrict__ gqdT,
                                             const T* __restrict__ gtraj, T* gq0, T* gqd0, T* gtau,
                                             T* gm_acc, T* ring) {
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const int nq = m.nqv[slot] & 0xffff, nv = m.nqv[slot] >> 16;
  const V3<T> g{m.g0, m.g1, m.g2};
  Sys<T> s = sys_of<T, SMEM, true>(m, slot);
  Col<T> gq{gq0 + b, B}, gqd{gqd0 + b, B};
  Col<T> gm{gm_acc + slot, B};
  T* sbuf = nullptr;  // [2][NX + nvm][LANES]: checkpointed state and tau, one step ahead
  if (SMEM) {  // state adjoint and mass-gradient sums on chip; written out at the end
    const SmemTile<T> st = smem_tile<T, true>(m.maxL, NX, nvm, slot % LANES);
    gq = Col<T>{st.state, LANES};
    gqd = Col<T>{st.state + nqm * LANES, LANES};
    gm = Col<T>{st.gm, LANES};
    sbuf = st.stream;
  }
  for (int d = 0; d < nqm; ++d) {
    T v = d < nq ? gqT[d * B + b] : T(0);
    if (gtraj && d < nq) v += gtraj[(Tn * NX + d) * B + b];
    gq[d] = v;
  }
  for (int d = 0; d < nvm; ++d) {
    T v = d < nv ? gqdT[d * B + b] : T(0);
    if (gtraj && d < nv) v += gtraj[(Tn * NX + nqm + d) * B + b];
    gqd[d] = v;
  }
  for (int l = 0; l < s.nl; ++l) gm[l] = T(0);
  const long long nseg = (Tn + k - 1) / k;
  if (SMEM && k == 1) {
    // every step has its own checkpoint: stream x^t and tau^t into shared memory,
    // fetching step t-1's while step t is differentiated
    const int W = NX + nvm;
    auto fetch = [&](long long t, int buf) {
      T* dst = sbuf + buf * W * LANES;
      for (int d = 0; d < NX; ++d) cp_async(dst + d * LANES, ckpt + (t * NX + d) * B + b);
      for (int d = 0; d < nvm; ++d) cp_async(dst + (NX + d) * LANES, tau + (t * nvm + d) * B + b);
    };
    if (Tn > 0) fetch(Tn - 1, (int)((Tn - 1) & 1));
    cp_commit();
    for (long long t = Tn - 1; t >= 0; --t) {
      if (t > 0) fetch(t - 1, (int)((t - 1) & 1));
      cp_commit();
      cp_wait_all_but_newest();
      const T* xb = sbuf + (t & 1) * W * LANES;
      Col<const T> q{xb, LANES}, qd{xb + nqm * LANES, LANES};
      aba_forward<T, DT, true>(s, q, qd, Col<const T>{xb + NX * LANES, LANES}, g);
      T* gt = gtau + t * nvm * B + b;
      step_adjoint<T, DT>(s, q, qd, gq, gqd, Col<T>{gt, B}, gm, g, m.dt, m.integ);
      for (int d = nv; d < nvm; ++d) gt[d * B] = T(0);
      if (gtraj) {
        const T* gx = gtraj + t * NX * B + b;
        for (int d = 0; d < nq; ++d) gq[d] += gx[d * B];
        for (int d = 0; d < nv; ++d) gqd[d] += gx[(nqm + d) * B];
      }
    }
    cp_wait_all();
  } else {
    for (long long seg = nseg - 1; seg >= 0; --seg) {
      const long long t0 = seg * k;
      const long long t1 = (t0 + k < Tn) ? t0 + k : Tn;
      const T* xs = ckpt + seg * NX * B + b;
      if (k > 1 && !m.quadratic) {  // replay the segment once, keeping its states (ring by slot)
        T* r0 = ring + slot;
        for (int d = 0; d < NX; ++d) r0[d * B] = xs[d * B];
        for (long long j = 1; j < t1 - t0; ++j) {
          const T* prev = ring + (j - 1) * NX * B + slot;
          T* cur = ring + j * NX * B + slot;
          for (int d = 0; d < NX; ++d) cur[d * B] = prev[d * B];
          aba_forward<T, DT, false>(s, Col<const T>{cur, B}, Col<const T>{cur + nqm * B, B},
                         Col<const T>{tau + (t0 + j - 1) * nvm * B + b, B}, g);
          integrate<T>(s, Col<T>{cur, B}, Col<T>{cur + nqm * B, B}, m.dt, m.integ);
        }
      }
      for (long long t = t1 - 1; t >= t0; --t) {
        const T* x = (k > 1) ? ring + (t - t0) * NX * B + slot : xs;
        if (k > 1 && m.quadratic) {  // recompute x^t from the segment checkpoint: t - t0 steps
          T* cur = ring + slot;
          x = cur;
          for (int d = 0; d < NX; ++d) cur[d * B] = xs[d * B];
          for (long long j = t0; j < t; ++j) {
            aba_forward<T, DT, false>(s, Col<const T>{cur, B}, Col<const T>{cur + nqm * B, B},
                                      Col<const T>{tau + j * nvm * B + b, B}, g);
            integrate<T>(s, Col<T>{cur, B}, Col<T>{cur + nqm * B, B}, m.dt, m.integ);
          }
        }
        Col<const T> q{x, B}, qd{x + nqm * B, B};
        aba_forward<T, DT, true>(s, q, qd, Col<const T>{tau + t * nvm * B + b, B}, g);
        T* gt = gtau + t * nvm * B + b;
        step_adjoint<T, DT>(s, q, qd, gq, gqd, Col<T>{gt, B}, gm, g, m.dt, m.integ);
        for (int d = nv; d < nvm; ++d) gt[d * B] = T(0);
        if (gtraj) {
          const T* gx = gtraj + t * NX * B + b;
          for (int d = 0; d < nq; ++d) gq[d] += gx[d * B];
          for (int d = 0; d < nv; ++d) gqd[d] += gx[(nqm + d) * B];
        }
      }
    }
  }
  bool ok = true;
  for (int d = 0; d < nq; ++d) ok &= finite_t(gq[d]);
  for (int d = 0; d < nv; ++d) ok &= finite_t(gqd[d]);
  for (int l = 0; l < s.nl; ++l) ok &= finite_t(gm[l]);
  if (!ok) m.status[b] |= 1;
  if (SMEM) {
    for (int d = 0; d < nqm; ++d) gq0[d * B + b] = gq[d];
    for (int d = 0; d < nvm; ++d) gqd0[d * B + b] = gqd[d];
    for (int l = 0; l < s.nl; ++l) gm_acc[l * B + slot] = gm[l];
  }
}

// Work distribution.  Grid mode: block i takes work unit i (blockDim slots).
// Persistent mode: a grid sized to the resident capacity, each block taking the
// next unit from an atomic counter until none is left (the counter is reset by
// the host before every launch; the loop ends after at most units + 1 tickets).
__device__ __forceinline__ int next_unit(unsigned* counter) {
  __shared__ int unit_s;
  if (threadIdx.x == 0) unit_s = (int)atomicAdd(counter, 1u);
  __syncthreads();
  const int unit = unit_s;
  __syncthreads();
  return unit;
}

#define ABASIM_FOR_EACH_SLOT(m, ...)                                         \
  int unit = (m).persistent ? next_unit((m).counter) : (int)blockIdx.x;      \
  while ((long long)unit * blockDim.x < (m).B) {                             \
    const int slot = unit * blockDim.x + threadIdx.x;                        \
    if (slot < (m).B) { __VA_ARGS__; }                                       \
    if (!(m).persistent) break;                                              \
    unit = next_unit((m).counter);                                           \
  }

template <class T, class DT, bool SMEM>
__global__ void k_rollout(DevModel<T> m, const T* __restrict__ q0, const T* __restrict__ qd0,
                          const T* __restrict__ tau, long long Tn, int k, T* ckpt, T* qT, T* qdT,
                          T* traj) {
  ABASIM_FOR_EACH_SLOT(m, rollout_one<T, DT, SMEM>(m, slot, q0, qd0, tau, Tn, k, ckpt, qT, qdT, traj))
}

template <class T, class DT, bool SMEM>
__global__ void k_backward(DevModel<T> m, const T* __restrict__ ckpt, const T* __restrict__ tau,
                           long long Tn, int k, const T* __restrict__ gqT, const T* __restrict__ gqdT,
                           const T* __restrict__ gtraj, T* gq0, T* gqd0, T* gtau, T* gm_acc,
                           T* ring) {
  ABASIM_FOR_EACH_SLOT(m, backward_one<T, DT, SMEM>(m, slot, ckpt, tau, Tn, k, gqT, gqdT, gtraj, gq0, gqd0,
                                          gtau, gm_acc, ring))
}

// One step with tangents: the state, torque and tape are dual numbers staged in
// the caller's workspace [tile][...][lane]; model constants stay plain.
template <class T, class DT>
__global__ void k_step_jvp(DevModel<T> m, const T* __restrict__ q, const T* __restrict__ qd,
                           const T* __restrict__ tau, const T* __restrict__ dq,
                           const T* __restrict__ dqd, const T* __restrict__ dtau, T* q_out,
                           T* qd_out, T* dq_out, T* dqd_out, Dual<T>* work) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= m.B) return;
  using D = Dual<T>;
  using DD = Dual<DT>;
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max;
  const long long tile = slot / LANES, lane = slot % LANES;
  const long long L = m.maxL;
  const long long per_tile = L * NTAPE + nqm + 2LL * nvm;  // tape, q, qd, tau
  D* base = work + tile * per_tile * LANES + lane;
  Sys<D, T> s{m.prm + tile * L * NPRM * LANES + lane, m.meta + tile * L * LANES + lane, base, nullptr,
              m.nl[slot]};
  Col<D> xq{base + L * NTAPE * LANES, LANES};
  Col<D> xqd{base + (L * NTAPE + nqm) * LANES, LANES};
  Col<D> xt{base + (L * NTAPE + nqm + nvm) * LANES, LANES};
  for (int d = 0; d < nqm; ++d) xq[d] = D(q[d * B + b], dq ? dq[d * B + b] : T(0));
  for (int d = 0; d < nvm; ++d) {
    xqd[d] = D(qd[d * B + b], dqd ? dqd[d * B + b] : T(0));
    xt[d] = D(tau[d * B + b], dtau ? dtau[d * B + b] : T(0));
  }
  const V3<D> g{D(m.g0), D(m.g1), D(m.g2)};
  static_assert(sizeof(DD) == 2 * sizeof(DT), "dual layout");
  aba_forward<D, D, false>(s, Col<const D>{xq.p, LANES}, Col<const D>{xqd.p, LANES},
                           Col<const D>{xt.p, LANES}, g);
  integrate<D>(s, xq, xqd, D(m.dt), m.integ);
  for (int d = 0; d < nqm; ++d) {
    q_out[d * B + b] = xq[d].v;
    dq_out[d * B + b] = xq[d].d;
  }
  for (int d = 0; d < nvm; ++d) {
    qd_out[d * B + b] = xqd[d].v;
    dqd_out[d * B + b] = xqd[d].d;
  }
}

template <class T>
__global__ void k_gather_mass_grad(const T* __restrict__ gm_acc, const int* __restrict__ link_slot,
                                   int L, T* gmass) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < L) gmass[j] = gm_acc[link_slot[j]];
}

template <class T>
__global__ void k_set_masses(T* prm, const int* __restrict__ link_slot, int L, long long B, int maxL,
                             const T* __restrict__ mass) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  const int ls = link_slot[j];
  const long long l = ls / B, slot = ls % B;
  const long long tile = slot / LANES, lane = slot % LANES;
  prm[((tile * maxL + l) * NPRM + P_M) * LANES + lane] = mass[j];
}

// ------------------------------------------------------------------ launches

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

// Grid size and mode of a batched launch; resets the ticket of persistent launches.
template <class K>
int launch_shape(sim_handle* h, K kernel, int* grid, int* persistent, size_t shm, void* stream) {
  const int units = (h->B + h->block - 1) / h->block;
  *grid = units;
  *persistent = 0;
  if (h->schedule != SIM_SCHED_PERSISTENT) return SIM_OK;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, h->block, shm);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
  const int cap = std::max(1, per_sm) * std::max(1, h->sms);
  *grid = std::min(units, cap);
  *persistent = 1;
  e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), S(stream));
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "work ticket reset");
}

// Dynamic shared memory for on-chip tapes (0 = keep them in global scratch):
// the block's tiles x links x fields, if it fits the per-block opt-in limit and,
// in auto mode, if the smaller residency it implies adds no wave of blocks over
// the global-tape kernel.
template <class T, class KS, class KG>
int smem_bytes(sim_handle* h, KS kernel_smem, KG kernel_global, bool bwd, size_t* bytes) {
  *bytes = 0;
  if (h->tape_space == SIM_TAPE_GLOBAL) return SIM_OK;
  const size_t need = (size_t)(h->block / LANES) *
                      smem_per_tile(h->maxL, h->nq_max + h->nv_max, h->nv_max, bwd) * LANES * sizeof(T);
  int limit = 0;
  cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
  if (need > (size_t)limit) {
    if (h->tape_space == SIM_TAPE_SHARED) return fail(h, SIM_EUNSUPPORTED, "tape does not fit in shared memory");
    return SIM_OK;
  }
  e = cudaFuncSetAttribute(kernel_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
  if (h->tape_space == SIM_TAPE_AUTO) {
    int per_sm_s = 0, per_sm_g = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, kernel_smem, h->block, need);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, kernel_global, h->block, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
    const long long units = (h->B + h->block - 1) / h->block;
    const long long sms = std::max(1, h->sms);
    const long long waves_s = per_sm_s > 0 ? (units + sms * per_sm_s - 1) / (sms * per_sm_s) : 1LL << 40;
    const long long waves_g = per_sm_g > 0 ? (units + sms * per_sm_g - 1) / (sms * per_sm_g) : 1LL << 40;
    if (waves_s > waves_g) return SIM_OK;
  }
  *bytes = need;
  return SIM_OK;
}

template <class T, class DT>
int launch_rollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T_,
                   int k, void* ckpt, void* qT, void* qdT, void* traj, void* stream) {
  DevModel<T> m = dev_model<T>(h);
  size_t shm = 0;
  int rc = SIM_OK;
  if (sizeof(T) == 4) rc = smem_bytes<T>(h, k_rollout<T, DT, true>, k_rollout<T, DT, false>, false, &shm);
  if (rc != SIM_OK) return rc;
  auto kern = shm ? k_rollout<T, DT, true> : k_rollout<T, DT, false>;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream);
  if (rc != SIM_OK) return rc;
  kern<<<grid, h->block, shm, S(stream)>>>(m, (const T*)q0, (const T*)qd0, (const T*)tau, (long long)T_,
                                           k, (T*)ckpt, (T*)qT, (T*)qdT, (T*)traj);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "rollout launch");
}

template <class T, class DT>
int launch_backward(sim_handle* h, const void* ckpt, const void* tau, int64_t T_, int k,
                    const void* gqT, const void* gqdT, const void* gtraj, void* gq0, void* gqd0,
                    void* gtau, void* gmass, void* work, void* stream) {
  DevModel<T> m = dev_model<T>(h);
  size_t shm = 0;
  int rc = SIM_OK;
  if (sizeof(T) == 4) rc = smem_bytes<T>(h, k_backward<T, DT, true>, k_backward<T, DT, false>, true, &shm);
  if (rc != SIM_OK) return rc;
  auto kern = shm ? k_backward<T, DT, true> : k_backward<T, DT, false>;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream);
  if (rc != SIM_OK) return rc;
  kern<<<grid, h->block, shm, S(stream)>>>(m, (const T*)ckpt, (const T*)tau, (long long)T_, k,
                                           (const T*)gqT, (const T*)gqdT, (const T*)gtraj, (T*)gq0,
                                           (T*)gqd0, (T*)gtau, (T*)h->gm_acc, (T*)work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
  if (gmass) {
    k_gather_mass_grad<T><<<(h->L_total + 255) / 256, 256, 0, S(stream)>>>(
        (const T*)h->gm_acc, h->link_slot, h->L_total, (T*)gmass);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "mass-gradient launch");
  }
  return SIM_OK;
}

bool is_fp64(const sim_handle* h) { return h->precision == SIM_FP64; }

// ------------------------------------------------------------------ validation

bool near(double a, double b, double tol) { return std::fabs(a - b) <= tol; }

int validate(const sim_model_desc* d, std::string& why) {
  auto bad = [&](const std::string& s) { why = s; return SIM_EINVAL; };
  if (!d) return bad("null model description");
  if (d->n_systems < 1) return bad("n_systems must be >= 1");
  if (d->precision < SIM_FP64 || d->precision > SIM_FP32_D64) return bad("unknown precision");
  if (d->integrator != SIM_SEMI_IMPLICIT_EULER && d->integrator != SIM_EXPLICIT_EULER)
    return bad("unknown integrator");
  if (!(d->dt > 0) || !std::isfinite(d->dt)) return bad("dt must be finite and > 0");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(d->gravity[i])) return bad("gravity must be finite");
  if (!d->sys_link_offset || !d->parent || !d->joint_type || !d->axis || !d->X_tree || !d->mass ||
      !d->com || !d->I_com)
    return bad("null model array");
  if (d->sys_link_offset[0] != 0) return bad("sys_link_offset[0] must be 0");
  for (int b = 0; b < d->n_systems; ++b) {
    const int o0 = d->sys_link_offset[b], o1 = d->sys_link_offset[b + 1];
    const int n = o1 - o0;
    char buf[160];
    if (n < 1 || n > kMaxLinks) {
      snprintf(buf, sizeof buf, "system %d has %d links (1..%d allowed)", b, n, kMaxLinks);
      return bad(buf);
    }
    int nq = 0, nv = 0;
    for (int l = 0; l < n; ++l) {
      const int i = o0 + l;
      const int p = d->parent[i], jt = d->joint_type[i];
      if (p < -1 || p >= l) {
        snprintf(buf, sizeof buf, "system %d link %d: parent %d not in [-1, %d)", b, l, p, l);
        return bad(buf);
      }
      if (jt == SIM_FREE) {
        if (l != 0 || p != -1) {
          snprintf(buf, sizeof buf, "system %d link %d: a free joint must be the first link", b, l);
          return bad(buf);
        }
        nq += 7; nv += 6;
      } else if (jt == SIM_REVOLUTE) {
        const double* a = d->axis + 3 * i;
        const double nn = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        if (!near(nn, 1.0, 1e-6)) {
          snprintf(buf, sizeof buf, "system %d link %d: axis is not unit length", b, l);
          return bad(buf);
        }
        nq += 1; nv += 1;
      } else {
        snprintf(buf, sizeof buf, "system %d link %d: unknown joint type %d", b, l, jt);
        return bad(buf);
      }
      const double* E = d->X_tree + 12 * i;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double s = 0;
          for (int x = 0; x < 3; ++x) s += E[3 * x + r] * E[3 * x + c];
          if (!near(s, r == c ? 1.0 : 0.0, 1e-6)) {
            snprintf(buf, sizeof buf, "system %d link %d: X_tree rotation is not orthonormal", b, l);
            return bad(buf);
          }
        }
      for (int x = 0; x < 12; ++x)
        if (!std::isfinite(E[x])) return bad("non-finite X_tree");
      const double m = d->mass[i];
      if (!(m > 0) || !std::isfinite(m)) {
        snprintf(buf, sizeof buf, "system %d link %d: mass must be finite and > 0", b, l);
        return bad(buf);
      }
      const double* Ic = d->I_com + 6 * i;
      for (int x = 0; x < 6; ++x)
        if (!std::isfinite(Ic[x]) || !std::isfinite(d->com[3 * i + x % 3]))
          return bad("non-finite inertia or COM");
      if (d->damping && (!(d->damping[i] >= 0) || !std::isfinite(d->damping[i]))) {
        snprintf(buf, sizeof buf, "system %d link %d: damping must be finite and >= 0", b, l);
        return bad(buf);
      }
      if (Ic[0] < 0 || Ic[1] < 0 || Ic[2] < 0) {
        snprintf(buf, sizeof buf, "system %d link %d: negative principal inertia", b, l);
        return bad(buf);
      }
    }
    if (nq > kMaxCoords || nv > kMaxCoords) return bad("too many coordinates in one system");
  }
  return SIM_OK;
}

template <class T> int upload(sim_handle* h, const std::vector<double>& prm_h) {
  std::vector<T> v(prm_h.begin(), prm_h.end());
  cudaError_t e = cudaMalloc(&h->prm, v.size() * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(h, e, "model upload");
  e = cudaMemcpy(h->prm, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "model upload");
  return SIM_OK;
}

int check_handle(const sim_handle* h) { return h ? SIM_OK : SIM_EINVAL; }

// ------------------------------------------------------------------ static scratch
// Per-link tape for sim_step_batch_static: a file-scope device array, so that
// entry point needs no allocation at all.  Every GPU that loads this library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_tape[SIM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_tape on the current device, looked up once per
// device (the symbol's name in host code is only a host-side stand-in).
int static_tape(sim_handle* h, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "static scratch: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(h, SIM_EUNSUPPORTED, "static scratch: device index too large");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_tape);
    if (e != cudaSuccess) return cuda_fail(h, e, "static scratch: cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SIM_OK;
}

template <class T, class DT>
int launch_step_static(sim_handle* h, const void* q, const void* qd, const void* tau, void* q_out,
                       void* qd_out, void* stream) {
  void* tape = nullptr;
  int rc = static_tape(h, &tape);
  if (rc != SIM_OK) return rc;
  DevModel<T> m = dev_model<T>(h);
  m.tape = (T*)tape;
  const int grid = (h->B + h->block - 1) / h->block;
  k_rollout<T, DT, false><<<grid, h->block, 0, S(stream)>>>(m, (const T*)q, (const T*)qd, (const T*)tau, 1LL, 1,
                                                  (T*)nullptr, (T*)q_out, (T*)qd_out, (T*)nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "static step launch");
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

int sim_create(const sim_model_desc* d, sim_handle** out) {
  if (!out) return fail(nullptr, SIM_EINVAL, "null output pointer");
  *out = nullptr;
  std::string why;
  if (validate(d, why) != SIM_OK) return fail(nullptr, SIM_EINVAL, why);
  sim_handle* h = new sim_handle();
  h->B = d->n_systems;
  h->precision = d->precision;
  h->integrator = d->integrator;
  h->dt = d->dt;
  for (int i = 0; i < 3; ++i) h->g[i] = d->gravity[i];
  h->scalar = h->precision == SIM_FP64 ? 8 : 4;
  h->L_total = d->sys_link_offset[h->B];
  cudaGetDevice(&h->device);
  const int B = h->B;
  std::vector<int> nl_sys(B);
  for (int b = 0; b < B; ++b) {
    nl_sys[b] = d->sys_link_offset[b + 1] - d->sys_link_offset[b];
    h->maxL = std::max(h->maxL, nl_sys[b]);
  }
  // slots: systems sorted by link count, longest first (stable), so a warp's
  // threads walk equally long link loops and the longest work starts first
  std::vector<int> order(B);
  for (int b = 0; b < B; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nl_sys[x] > nl_sys[y]; });
  h->h_sys_of_slot = order;
  const int maxL = h->maxL;
  const size_t Bpad = (size_t)((B + LANES - 1) / LANES) * LANES;
  h->Bpad = (int)Bpad;
  std::vector<int> nl(B), nqv(B);
  std::vector<double> prm((size_t)maxL * NPRM * Bpad, 0.0);
  std::vector<int> meta((size_t)maxL * Bpad, 0), slot(h->L_total);
  for (int sl = 0; sl < B; ++sl) {
    const int b = order[sl];
    nl[sl] = nl_sys[b];
    int qo = 0, vo = 0;
    for (int l = 0; l < nl[sl]; ++l) {
      const int i = d->sys_link_offset[b] + l;
      const int jt = d->joint_type[i];
      const size_t tile = sl / LANES, lane = sl % LANES;
      auto P = [&](int f) -> double& { return prm[((tile * maxL + l) * NPRM + f) * LANES + lane]; };
      for (int x = 0; x < 12; ++x) P(P_E + x) = d->X_tree[12 * i + x];
      for (int x = 0; x < 3; ++x) {
        P(P_AX + x) = jt == SIM_REVOLUTE ? d->axis[3 * i + x] : 0.0;
        P(P_C + x) = d->com[3 * i + x];
      }
      P(P_M) = d->mass[i];
      for (int x = 0; x < 6; ++x) P(P_IC + x) = d->I_com[6 * i + x];
      P(P_DAMP) = (d->damping && jt == SIM_REVOLUTE) ? d->damping[i] : 0.0;
      bool treechild = false;  // a child other than link l + 1
      for (int c = l + 2; c < nl[sl]; ++c)
        if (d->parent[d->sys_link_offset[b] + c] == l) treechild = true;
      meta[(tile * maxL + l) * LANES + lane] = make_meta(d->parent[i], jt, treechild, qo, vo);
      slot[i] = l * B + sl;
      qo += jt == SIM_FREE ? 7 : 1;
      vo += jt == SIM_FREE ? 6 : 1;
    }
    nqv[sl] = qo | (vo << 16);
    h->nq_max = std::max(h->nq_max, qo);
    h->nv_max = std::max(h->nv_max, vo);
  }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  int rc = h->precision == SIM_FP64 ? upload<double>(h, prm) : upload<float>(h, prm);
  auto alloc = [&](void** p, size_t bytes, const char* what) -> int {
    cudaError_t e = cudaMalloc(p, bytes);
    return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, what);
  };
  auto put = [&](void* dst, const void* src, size_t bytes) -> int {
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "model upload");
  };
  if (rc == SIM_OK) rc = alloc((void**)&h->meta, meta.size() * sizeof(int), "meta");
  if (rc == SIM_OK) rc = put(h->meta, meta.data(), meta.size() * sizeof(int));
  if (rc == SIM_OK) rc = alloc((void**)&h->nl, B * sizeof(int), "nl");
  if (rc == SIM_OK) rc = put(h->nl, nl.data(), B * sizeof(int));
  if (rc == SIM_OK) rc = alloc((void**)&h->nqv, B * sizeof(int), "nqv");
  if (rc == SIM_OK) rc = put(h->nqv, nqv.data(), B * sizeof(int));
  if (rc == SIM_OK) rc = alloc((void**)&h->link_slot, slot.size() * sizeof(int), "link map");
  if (rc == SIM_OK) rc = put(h->link_slot, slot.data(), slot.size() * sizeof(int));
  if (rc == SIM_OK) rc = alloc(&h->tape, (size_t)maxL * NTAPE * Bpad * h->scalar, "tape");
  if (rc == SIM_OK) rc = alloc(&h->adj, (size_t)maxL * NADJ * Bpad * h->scalar, "adjoint tape");
  if (rc == SIM_OK) rc = alloc(&h->gm_acc, (size_t)maxL * B * h->scalar, "mass-gradient buffer");
  if (rc == SIM_OK) rc = alloc((void**)&h->status, B * sizeof(int), "status");
  if (rc == SIM_OK) rc = alloc((void**)&h->sys_of_slot, B * sizeof(int), "slot order");
  if (rc == SIM_OK) rc = put(h->sys_of_slot, order.data(), B * sizeof(int));
  if (rc == SIM_OK) rc = alloc((void**)&h->counter, sizeof(unsigned), "work ticket");
  if (rc == SIM_OK) {
    cudaError_t e = cudaMemset(h->status, 0, B * sizeof(int));
    if (e != cudaSuccess) rc = cuda_fail(h, e, "status init");
  }
  if (rc != SIM_OK) {
    g_create_error = h->err;
    sim_destroy(h);
    return rc;
  }
  *out = h;
  return SIM_OK;
}

void sim_destroy(sim_handle* h) {
  if (!h) return;
  void* ptrs[] = {h->prm, h->meta, h->nl, h->nqv, h->tape, h->adj, h->gm_acc, h->link_slot,
                  h->status, h->sys_of_slot, h->counter};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

int sim_dims(const sim_handle* h, int32_t* n_systems, int32_t* nq_max, int32_t* nv_max,
             int32_t* n_links_total) {
  if (!h) return SIM_EINVAL;
  if (n_systems) *n_systems = h->B;
  if (nq_max) *nq_max = h->nq_max;
  if (nv_max) *nv_max = h->nv_max;
  if (n_links_total) *n_links_total = h->L_total;
  return SIM_OK;
}

size_t sim_ckpt_bytes(const sim_handle* h, int64_t T, int32_t k) {
  if (!h || T < 0 || k < 1) return 0;
  const int64_t n = (T + k - 1) / k;
  return (size_t)n * (h->nq_max + h->nv_max) * h->B * h->scalar;
}

size_t sim_work_bytes(const sim_handle* h, int32_t k) {
  if (!h || k <= 1) return 0;
  return (size_t)k * (h->nq_max + h->nv_max) * h->B * h->scalar;
}

int sim_set_masses(sim_handle* h, const void* mass, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!mass) return fail(h, SIM_EINVAL, "null mass array");
  const int grid = (h->L_total + 255) / 256;
  if (is_fp64(h))
    k_set_masses<double><<<grid, 256, 0, S(stream)>>>((double*)h->prm, h->link_slot, h->L_total,
                                                      h->B, h->maxL, (const double*)mass);
  else
    k_set_masses<float><<<grid, 256, 0, S(stream)>>>((float*)h->prm, h->link_slot, h->L_total,
                                                     h->B, h->maxL, (const float*)mass);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "set_masses launch");
}

int sim_rollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T,
                int32_t k, void* ckpt, void* qT, void* qdT, void* traj, void* stream) {
  if (!h) return SIM_EINVAL;
  if (T < 0 || k < 1) return fail(h, SIM_EINVAL, "need T >= 0 and k >= 1");
  if (!q0 || !qd0 || !qT || !qdT || (T > 0 && !tau))
    return fail(h, SIM_EINVAL, "null state or torque pointer");
  switch (h->precision) {
    case SIM_FP64: return launch_rollout<double, double>(h, q0, qd0, tau, T, k, ckpt, qT, qdT, traj, stream);
    case SIM_FP32: return launch_rollout<float, float>(h, q0, qd0, tau, T, k, ckpt, qT, qdT, traj, stream);
    default: return launch_rollout<float, double>(h, q0, qd0, tau, T, k, ckpt, qT, qdT, traj, stream);
  }
}

int sim_step_batch(sim_handle* h, const void* q, const void* qd, const void* tau, void* q_out,
                   void* qd_out, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!tau) return fail(h, SIM_EINVAL, "null torque pointer");
  return sim_rollout(h, q, qd, tau, 1, 1, nullptr, q_out, qd_out, nullptr, stream);
}

int sim_step_batch_static(sim_handle* h, const void* q, const void* qd, const void* tau,
                          void* q_out, void* qd_out, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!q || !qd || !tau || !q_out || !qd_out) return fail(h, SIM_EINVAL, "null state or torque pointer");
  const size_t need = (size_t)h->maxL * NTAPE * h->Bpad * h->scalar;
  if (need > (size_t)SIM_STATIC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf, "batch needs %zu bytes of step scratch; the static array holds %zu",
             need, (size_t)SIM_STATIC_SCRATCH_BYTES);
    return fail(h, SIM_ENOMEM, buf);
  }
  switch (h->precision) {
    case SIM_FP64: return launch_step_static<double, double>(h, q, qd, tau, q_out, qd_out, stream);
    case SIM_FP32: return launch_step_static<float, float>(h, q, qd, tau, q_out, qd_out, stream);
    default: return launch_step_static<float, double>(h, q, qd, tau, q_out, qd_out, stream);
  }
}

size_t sim_jvp_work_bytes(const sim_handle* h) {
  if (!h) return 0;
  const size_t per_tile = (size_t)h->maxL * NTAPE + h->nq_max + 2 * (size_t)h->nv_max;
  return per_tile * h->Bpad * 2 * h->scalar;
}

int sim_step_jvp(sim_handle* h, const void* q, const void* qd, const void* tau, const void* dq,
                 const void* dqd, const void* dtau, void* q_out, void* qd_out, void* dq_out,
                 void* dqd_out, void* work, size_t work_bytes, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!q || !qd || !tau || !q_out || !qd_out || !dq_out || !dqd_out)
    return fail(h, SIM_EINVAL, "null state, torque or output pointer");
  if (!work || work_bytes < sim_jvp_work_bytes(h))
    return fail(h, SIM_ENOMEM, "workspace smaller than sim_jvp_work_bytes");
  const int grid = (h->B + h->block - 1) / h->block;
  switch (h->precision) {
    case SIM_FP64:
      k_step_jvp<double, double><<<grid, h->block, 0, S(stream)>>>(
          dev_model<double>(h), (const double*)q, (const double*)qd, (const double*)tau,
          (const double*)dq, (const double*)dqd, (const double*)dtau, (double*)q_out,
          (double*)qd_out, (double*)dq_out, (double*)dqd_out, (Dual<double>*)work);
      break;
    default:
      k_step_jvp<float, float><<<grid, h->block, 0, S(stream)>>>(
          dev_model<float>(h), (const float*)q, (const float*)qd, (const float*)tau,
          (const float*)dq, (const float*)dqd, (const float*)dtau, (float*)q_out, (float*)qd_out,
          (float*)dq_out, (float*)dqd_out, (Dual<float>*)work);
      break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "jvp launch");
}

int sim_backward_rollout(sim_handle* h, const void* ckpt, const void* tau, int64_t T, int32_t k,
                         const void* gqT, const void* gqdT, const void* g_traj, void* gq0,
                         void* gqd0, void* gtau, void* gmass, void* work, size_t work_bytes,
                         void* stream) {
  if (!h) return SIM_EINVAL;
  if (T < 0 || k < 1) return fail(h, SIM_EINVAL, "need T >= 0 and k >= 1");
  if (!gqT || !gqdT || !gq0 || !gqd0 || (T > 0 && (!ckpt || !tau || !gtau)))
    return fail(h, SIM_EINVAL, "null pointer argument");
  if (k > 1 && T > 0 && (!work || work_bytes < sim_work_bytes(h, k)))
    return fail(h, SIM_ENOMEM, "workspace smaller than sim_work_bytes(k)");
  switch (h->precision) {
    case SIM_FP64:
      return launch_backward<double, double>(h, ckpt, tau, T, k, gqT, gqdT, g_traj, gq0, gqd0, gtau, gmass, work, stream);
    case SIM_FP32:
      return launch_backward<float, float>(h, ckpt, tau, T, k, gqT, gqdT, g_traj, gq0, gqd0, gtau, gmass, work, stream);
    default:
      return launch_backward<float, double>(h, ckpt, tau, T, k, gqT, gqdT, g_traj, gq0, gqd0, gtau, gmass, work, stream);
  }
}

int sim_status(sim_handle* h, int32_t* flags) {
  if (!h) return SIM_EINVAL;
  std::vector<int32_t> tmp(h->B);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(tmp.data(), h->status, h->B * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  bool any = false;
  for (int b = 0; b < h->B; ++b) any |= tmp[b] != 0;
  if (flags) memcpy(flags, tmp.data(), h->B * sizeof(int32_t));
  return any ? SIM_ENONFINITE : SIM_OK;
}

int sim_clear_status(sim_handle* h, void* stream) {
  if (!h) return SIM_EINVAL;
  cudaError_t e = cudaMemsetAsync(h->status, 0, h->B * sizeof(int), S(stream));
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "status clear");
}

int sim_set_launch(sim_handle* h, int32_t threads, int32_t schedule) {
  if (!h) return SIM_EINVAL;
  if (schedule != SIM_SCHED_GRID && schedule != SIM_SCHED_PERSISTENT)
    return fail(h, SIM_EINVAL, "unknown schedule");
  if (threads == 0) threads = kDefaultBlock;
  if (threads < 32 || threads > 1024 || threads % 32)
    return fail(h, SIM_EINVAL, "block size must be a multiple of 32 in [32, 1024]");
  h->block = threads;
  h->schedule = schedule;
  return SIM_OK;
}

int sim_set_tape_space(sim_handle* h, int32_t space) {
  if (!h) return SIM_EINVAL;
  if (space != SIM_TAPE_AUTO && space != SIM_TAPE_GLOBAL && space != SIM_TAPE_SHARED)
    return fail(h, SIM_EINVAL, "unknown tape space");
  h->tape_space = space;
  return SIM_OK;
}

int sim_set_replay(sim_handle* h, int32_t mode) {
  if (!h) return SIM_EINVAL;
  if (mode != SIM_REPLAY_SEGMENT && mode != SIM_REPLAY_QUADRATIC) return fail(h, SIM_EINVAL, "unknown replay mode");
  h->replay = mode;
  return SIM_OK;
}

int sim_slot_order(const sim_handle* h, int32_t* sys_of_slot) {
  if (!h || !sys_of_slot) return SIM_EINVAL;
  memcpy(sys_of_slot, h->h_sys_of_slot.data(), h->B * sizeof(int32_t));
  return SIM_OK;
}

const char* sim_last_error(const sim_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
