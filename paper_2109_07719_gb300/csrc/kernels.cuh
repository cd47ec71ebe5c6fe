// Batched rollout / adjoint / JVP kernels and their launch functions (templated;
// instantiated per precision in inst_*.cu).  Thread i of a launch handles slot i;
// slots hold the systems sorted by link count (longest first); model constants
// and tapes are stored by slot in 32-system tiles, the caller's arrays by system.
#pragma once

#include <algorithm>
#include <type_traits>

#include "contact.cuh"
#include "dual.cuh"
#include "handle.h"

namespace abasim {
namespace host {

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
  T* ctape;  // per-link contact tape [tile][maxL][NCT][lane] (null: no contact spheres or limits)
  T* csys;   // per-system contact record [tile][NCS][lane]
  ContactParams<T> cp;
  double dt64;   // the time step in FP64
  double* x64;   // FP64 running state [nq_max + nv_max][B] of the rollout (null: off; FP32 + FP64 D only)
  int pf;        // world-aligned kernels with a global tape: prefetch distance in links (0: none)
  T* stk;        // world-aligned kernels: two stacks of parent values [2][tiles][wdepth][WSW][lane] (null: none)
  int wdepth;    // entries per stack
};

template <class T> DevModel<T> dev_model(const sim_handle* h) {
  return DevModel<T>{(const T*)h->prm, h->meta, h->nl, h->nqv, (T*)h->tape, (T*)h->adj, h->status,
                     h->sys_of_slot, h->counter, (long long)h->B, h->maxL, h->nq_max, h->nv_max, (T)h->dt,
                     (T)h->g[0], (T)h->g[1], (T)h->g[2], h->integrator, 0, 0,
                     h->replay == SIM_REPLAY_QUADRATIC, (T*)h->ctape, (T*)h->csys,
                     ContactParams<T>{(T)h->friction, (T)h->erp, h->pgs_iterations}, h->dt,
                     h->state64 ? (double*)h->x64 : nullptr, h->prefetch, (T*)h->wstk, h->wdepth};
}

extern __shared__ __align__(16) unsigned char g_smem[];

// Storage modes of the batched kernels: everything per system in global memory
// (ST_GLOBAL); tape and model constants global but the working state and the
// prefetched input streams on chip (ST_HYBRID); everything on chip (ST_SMEM);
// the two-warp pipelined adjoint (ST_PIPE, k_backward_pipe).
enum : int { ST_GLOBAL = 0, ST_HYBRID = 1, ST_SMEM = 2, ST_PIPE = 3 };

// Scalars per tile (32 systems) a kernel keeps in dynamic shared memory when it
// runs with on-chip storage: the tape (and, for the adjoint, its accumulators and
// the per-link mass-gradient sums), the tile's model constants and meta words,
// its working state (x for the forward rollout, the state adjoint for the
// backward one) and a double buffer for the per-step input streams (tau, plus the
// checkpointed state for the adjoint) fetched one step ahead.
__host__ __device__ __forceinline__ long long smem_per_tile(int maxL, int nx, int nv, bool bwd, int st) {
  if (st == ST_GLOBAL) return 0;
  const long long streams = nx + 2LL * (nv + (bwd ? nx : 0)) + (bwd ? maxL : 0);  // state, buffers, gm
  if (st == ST_HYBRID) return streams;
  return (long long)maxL * (NTAPE + NPRM + 1 + (bwd ? NADJ : 0)) + streams;
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

template <class T, bool BWD, int ST>
__device__ __forceinline__ SmemTile<T> smem_tile(int maxL, int nx, int nv, int lane) {
  const int tb = threadIdx.x / LANES;
  const long long L = maxL;
  T* base = reinterpret_cast<T*>(g_smem) + (long long)tb * smem_per_tile(maxL, nx, nv, BWD, ST) * LANES + lane;
  SmemTile<T> t{};
  if (ST == ST_SMEM) {
    t.tape = base;
    base += L * NTAPE * LANES;
    t.adj = base;
    if (BWD) base += L * NADJ * LANES;
    t.prm = base;
    base += L * NPRM * LANES;
    t.meta = reinterpret_cast<int*>(base);  // one scalar slot per int (T is 4 or 8 bytes)
    base += L * LANES;
  }
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
// 16-byte copy bypassing L1 (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_newest() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// With SMEM the tile's tape, constants, meta words and working state live in
// shared memory (copied in here); otherwise the tapes are in the handle's global
// scratch and the constants are read from global memory.
template <class T, int ST, bool BWD>
__device__ __forceinline__ Sys<T> sys_of(const DevModel<T>& m, int slot) {
  const long long tile = slot / LANES, lane = slot % LANES;
  const long long L = m.maxL;
  const T* gprm = m.prm + tile * L * NPRM * LANES + lane;
  const int* gmeta = m.meta + tile * L * LANES + lane;
  if (ST == ST_SMEM) {
    const SmemTile<T> st = smem_tile<T, BWD, ST>(m.maxL, m.nq_max + m.nv_max, m.nv_max, (int)lane);
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

template <class T> __device__ __forceinline__ CView<T> cview_of(const DevModel<T>& m, int slot) {
  const long long tile = slot / LANES, lane = slot % LANES;
  return CView<T>{m.ctape + tile * m.maxL * NCT * LANES + lane, m.csys + tile * NCS * LANES + lane};
}

// One step x -> x' in place: ABA, the contact and joint-limit impulses (CT: the
// model has contact spheres or joint limits), integration.
template <class T, class DT, bool CT>
__device__ __forceinline__ void forward_step(const DevModel<T>& m, const Sys<T>& s, int slot, Col<T> q,
                                             Col<T> qd, Col<const T> tau_t, V3<T> g,
                                             Col<double> xw = Col<double>{nullptr, 0}) {
  aba_forward<T, DT, false>(s, Col<const T>{q.p, q.B}, Col<const T>{qd.p, qd.B}, tau_t, g);
  const T* ct = nullptr;
  if constexpr (CT) {
    const CView<T> cv = cview_of(m, slot);
    const int nc =
        contact_forward<T, DT, T>(s, cv, Col<const T>{q.p, q.B}, Col<const T>{qd.p, qd.B}, m.dt, m.cp);
    if (nc > 0) ct = cv.ct;
  }
  if constexpr (!std::is_same<T, DT>::value) {
    if (xw.p) {  // the running state in FP64 (xw); the dynamics read its FP32 rounding
      const Col<double> xq = xw, xqd{xw.p + (long long)m.nq_max * xw.B, xw.B};
      integrate_in<double>(s, xq, xqd, m.dt64, m.integ, ct);
      for (int d = 0; d < m.nq_max; ++d) q[d] = (T)xq[d];
      for (int d = 0; d < m.nv_max; ++d) qd[d] = (T)xqd[d];
      return;
    }
  }
  integrate<T>(s, q, qd, m.dt, m.integ, ct);
}

// Recomputes the step from x^t and pulls the state adjoint (gq, gqd) back
// through it.  With active contact or limit rows the integrator adjoint runs
// first for every link (the constraint adjoint needs all of qdd's adjoint), then
// the constraint adjoint, then the ABA adjoint with its terms added.
template <class T, class DT, bool CT>
__device__ __forceinline__ void adjoint_step(const DevModel<T>& m, const Sys<T>& s, int slot, Col<const T> q,
                                             Col<const T> qd, Col<const T> tau_t, Col<T> gq, Col<T> gqd,
                                             Col<T> gt, Col<T> gm, V3<T> g) {
  aba_forward<T, DT, true>(s, q, qd, tau_t, g);
  if constexpr (CT) {
    const CView<T> cv = cview_of(m, slot);
    const int nc = contact_forward<T, DT, T>(s, cv, q, qd, m.dt, m.cp);
    if (nc > 0) {
      for (int l = 0; l < s.nl; ++l) {
        const int mt = s.M(l);
        T qb[6] = {0, 0, 0, 0, 0, 0};
        integrator_adjoint(s, l, meta_jtype(mt), meta_qoff(mt), meta_voff(mt), q, qd, gq, gqd, m.dt, m.integ,
                           qb, (const T*)cv.ct);
        for (int i = 0; i < 6; ++i) cv.L(l, C_QDDB + i) = qb[i];
      }
      contact_adjoint<T, DT, T>(s, cv, m.dt, m.cp);
      step_adjoint<T, DT>(s, q, qd, gq, gqd, gt, gm, g, m.dt, m.integ, (const T*)cv.ct);
      return;
    }
  }
  step_adjoint<T, DT>(s, q, qd, gq, gqd, gt, gm, g, m.dt, m.integ);
}

// ------------------------------------------------------------------ kernels
// Thread i of the launch handles slot i.  Slots hold the systems sorted by link
// count (longest first) so a warp's systems walk the same number of links; the
// model constants and tapes are stored by slot, the caller's arrays by system.

// T steps of one system.  The working state lives in (qT, qdT); checkpoints every
// k steps; optional full trajectory.
template <class T, class DT, int ST, bool CT>
__device__ __forceinline__ void rollout_one(const DevModel<T>& m, int slot, const T* __restrict__ q0,
                                            const T* __restrict__ qd0, const T* __restrict__ tau,
                                            long long Tn, int k, T* ckpt, T* qT, T* qdT, T* traj) {
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const V3<T> g{m.g0, m.g1, m.g2};
  constexpr bool SMEM = ST != ST_GLOBAL;  // on-chip state and streams
  Sys<T> s = sys_of<T, ST, false>(m, slot);
  Col<T> q{qT + b, B}, qd{qdT + b, B};
  T* sbuf = nullptr;  // [2][nvm][LANES] double buffer for tau
  if (SMEM) {  // the working state on chip; written to (qT, qdT) at the end
    const SmemTile<T> st = smem_tile<T, false, ST>(m.maxL, NX, nvm, slot % LANES);
    q = Col<T>{st.state, LANES};
    qd = Col<T>{st.state + nqm * LANES, LANES};
    sbuf = st.stream;
    if (Tn > 0)
      for (int d = 0; d < nvm; ++d) cp_async(sbuf + d * LANES, tau + (long long)d * B + b);
    cp_commit();
  }
  for (int d = 0; d < nqm; ++d) q[d] = q0[d * B + b];
  for (int d = 0; d < nvm; ++d) qd[d] = qd0[d * B + b];
  Col<double> xw{nullptr, 0};
  if constexpr (!std::is_same<T, DT>::value) {
    if (m.x64) {  // FP64 state accumulation, started from the FP32 initial state
      xw = Col<double>{m.x64 + b, B};
      for (int d = 0; d < nqm; ++d) xw[d] = (double)q[d];
      for (int d = 0; d < nvm; ++d) xw[nqm + d] = (double)qd[d];
    }
  }
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
    forward_step<T, DT, CT>(m, s, slot, q, qd, tau_t, g, xw);
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
template <class T, class DT, int ST, bool CT>
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
  constexpr bool SMEM = ST != ST_GLOBAL;  // on-chip state and streams
  Sys<T> s = sys_of<T, ST, true>(m, slot);
  Col<T> gq{gq0 + b, B}, gqd{gqd0 + b, B};
  Col<T> gm{gm_acc + slot, B};
  T* sbuf = nullptr;  // [2][NX + nvm][LANES]: checkpointed state and tau, one step ahead
  if (SMEM) {  // state adjoint and mass-gradient sums on chip; written out at the end
    const SmemTile<T> st = smem_tile<T, true, ST>(m.maxL, NX, nvm, slot % LANES);
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
      T* gt = gtau + t * nvm * B + b;
      adjoint_step<T, DT, CT>(m, s, slot, q, qd, Col<const T>{xb + NX * LANES, LANES}, gq, gqd, Col<T>{gt, B}, gm, g);
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
          forward_step<T, DT, CT>(m, s, slot, Col<T>{cur, B}, Col<T>{cur + nqm * B, B},
                              Col<const T>{tau + (t0 + j - 1) * nvm * B + b, B}, g);
        }
      }
      for (long long t = t1 - 1; t >= t0; --t) {
        const T* x = (k > 1) ? ring + (t - t0) * NX * B + slot : xs;
        if (k > 1 && m.quadratic) {  // recompute x^t from the segment checkpoint: t - t0 steps
          T* cur = ring + slot;
          x = cur;
          for (int d = 0; d < NX; ++d) cur[d * B] = xs[d * B];
          for (long long j = t0; j < t; ++j) {
            forward_step<T, DT, CT>(m, s, slot, Col<T>{cur, B}, Col<T>{cur + nqm * B, B},
                                Col<const T>{tau + j * nvm * B + b, B}, g);
          }
        }
        Col<const T> q{x, B}, qd{x + nqm * B, B};
        T* gt = gtau + t * nvm * B + b;
        adjoint_step<T, DT, CT>(m, s, slot, q, qd, Col<const T>{tau + t * nvm * B + b, B}, gq, gqd, Col<T>{gt, B},
                            gm, g);
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

// CT: the model has contact spheres or joint limits (a separate instantiation, so
// the kernels of unconstrained models carry none of the constraint code).
template <class T, class DT, int ST, bool CT = false>
__global__ void k_rollout(DevModel<T> m, const T* __restrict__ q0, const T* __restrict__ qd0,
                          const T* __restrict__ tau, long long Tn, int k, T* ckpt, T* qT, T* qdT,
                          T* traj) {
  ABASIM_FOR_EACH_SLOT(m, rollout_one<T, DT, ST, CT>(m, slot, q0, qd0, tau, Tn, k, ckpt, qT, qdT, traj))
}

template <class T, class DT, int ST, bool CT = false>
__global__ void k_backward(DevModel<T> m, const T* __restrict__ ckpt, const T* __restrict__ tau,
                           long long Tn, int k, const T* __restrict__ gqT, const T* __restrict__ gqdT,
                           const T* __restrict__ gtraj, T* gq0, T* gqd0, T* gtau, T* gm_acc,
                           T* ring) {
  ABASIM_FOR_EACH_SLOT(m, backward_one<T, DT, ST, CT>(m, slot, ckpt, tau, Tn, k, gqT, gqdT, gtraj, gq0, gqd0,
                                              gtau, gm_acc, ring))
}

}  // namespace host
}  // namespace abasim

#include "wkernels.cuh"

namespace abasim {
namespace host {

// ------------------------------------------------------------------ pipelined adjoint
// Two warps per 32-system tile, for batches of serial revolute chains with a
// checkpoint every step: the producer warp recomputes step t's forward
// intermediates from the checkpoint x^t into one of two shared-memory tapes
// (compact layout LAY_PROD) while the consumer warp runs the adjoint of step t + 1
// from the other one, with compact adjoint accumulators (LAY_CONS).  Step t's
// recompute does not depend on step t + 1's adjoint, so the two overlap.  Tape b
// holds the steps of parity b.  Hand-off by named barriers (hardware barriers: no
// spinning), one pair per tape: FULL(b) (the producer arrives when tape b holds
// its step, the consumer waits) and EMPTY(b) (the consumer arrives when it has
// finished a step from tape b that the producer will reuse, the producer waits
// before overwriting).  Per tile and tape both warps execute the same number of
// operations whatever their systems (inactive lanes included), and neither
// arrives twice at a barrier before the other's matching wait: the producer's
// next arrival at FULL(b) follows its wait on EMPTY(b), which follows the
// consumer's wait on FULL(b), and vice versa.
__device__ __forceinline__ void pair_sync_full(int b) {
  if (b) asm volatile("bar.sync 2, 64;\n" ::: "memory");
  else asm volatile("bar.sync 1, 64;\n" ::: "memory");
}
__device__ __forceinline__ void pair_arrive_full(int b) {
  if (b) asm volatile("bar.arrive 2, 64;\n" ::: "memory");
  else asm volatile("bar.arrive 1, 64;\n" ::: "memory");
}
__device__ __forceinline__ void pair_sync_empty(int b) {
  if (b) asm volatile("bar.sync 4, 64;\n" ::: "memory");
  else asm volatile("bar.sync 3, 64;\n" ::: "memory");
}
__device__ __forceinline__ void pair_arrive_empty(int b) {
  if (b) asm volatile("bar.arrive 4, 64;\n" ::: "memory");
  else asm volatile("bar.arrive 3, 64;\n" ::: "memory");
}

// Shared memory of one pipelined block, in scalars per lane: the two tapes, the
// adjoint accumulators, model constants, meta words, the state adjoint, the
// mass-gradient sums, the consumer's copy of x^t and the producer's
// double-buffered (x^t, tau^t) fetched one step ahead.
__host__ __device__ __forceinline__ long long pipe_smem_per_tile(int maxL, int nx, int nv) {
  return (long long)maxL * (2 * NTAPE_PROD + NADJ_CONS + NPRM + 1 + 1) + 2LL * nx + 2LL * (nx + nv);
}

template <class T, class DT>
__global__ void __launch_bounds__(2 * LANES, 1)
k_backward_pipe(DevModel<T> m, const T* __restrict__ ckpt, const T* __restrict__ tau, long long Tn, int k,
                const T* __restrict__ gqT, const T* __restrict__ gqdT, const T* __restrict__ gtraj, T* gq0,
                T* gqd0, T* gtau, T* gm_acc, T* ring) {
  const int warp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const bool consumer = warp == 0;
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const long long L = m.maxL;
  const V3<T> g{m.g0, m.g1, m.g2};
  constexpr int MS = (int)(sizeof(T) / sizeof(int));
  T* s_tape = reinterpret_cast<T*>(g_smem);  // [2][L][NTAPE_PROD][LANES]
  T* s_adj = s_tape + 2 * L * NTAPE_PROD * LANES;
  T* s_prm = s_adj + L * NADJ_CONS * LANES;
  T* s_meta = s_prm + L * NPRM * LANES;
  T* s_state = s_meta + L * LANES;
  T* s_gm = s_state + (long long)NX * LANES;
  T* s_x = s_gm + L * LANES;
  T* s_in = s_x + (long long)NX * LANES;  // [2][NX + nvm][LANES]
  const int W = NX + nvm;
  int* meta_l = reinterpret_cast<int*>(s_meta + lane);
  int unit = m.persistent ? next_unit(m.counter) : (int)blockIdx.x;
  while ((long long)unit * LANES < B) {
    const int slot = unit * LANES + lane;
    const bool act = slot < B;
    const int b = act ? m.sys_of_slot[slot] : 0;
    const int nl = act ? m.nl[slot] : 0;
    const int nq = act ? (m.nqv[slot] & 0xffff) : 0, nv = act ? (m.nqv[slot] >> 16) : 0;
    if (consumer && act) {
      const T* gprm = m.prm + (long long)unit * L * NPRM * LANES + lane;
      const int* gmeta = m.meta + (long long)unit * L * LANES + lane;
      for (int l = 0; l < nl; ++l) {
        for (int f = 0; f < NPRM; ++f) s_prm[(l * NPRM + f) * LANES + lane] = gprm[(l * NPRM + f) * LANES];
        meta_l[l * LANES * MS] = gmeta[l * LANES];
      }
    }
    __syncthreads();
    const T* sprm = s_prm + lane;
    // the producer's inputs of step t: x^t and tau^t, fetched one step ahead
    auto fetch = [&](long long t, int buf) {
      T* dst = s_in + buf * W * LANES + lane;
      for (int d = 0; d < NX; ++d) cp_async(dst + d * LANES, ckpt + (t * NX + d) * B + b);
      for (int d = 0; d < nvm; ++d) cp_async(dst + (NX + d) * LANES, tau + (t * nvm + d) * B + b);
    };
    if (!consumer) {
      if (act && Tn > 0) fetch(Tn - 1, (int)((Tn - 1) & 1));
      cp_commit();
    }
    Col<T> gq{s_state + lane, LANES}, gqd{s_state + nqm * LANES + lane, LANES}, gm{s_gm + lane, LANES};
    if (consumer && act) {
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
      for (int l = 0; l < nl; ++l) gm[l] = T(0);
    }
    for (long long t = Tn - 1; t >= 0; --t) {
      const int buf = (int)(t & 1);
      T* tape_b = s_tape + buf * L * NTAPE_PROD * LANES;
      if (!consumer) {  // producer: recompute step t into tape t & 1
        if (act && t > 0) fetch(t - 1, (int)((t - 1) & 1));
        cp_commit();
        cp_wait_all_but_newest();
        __syncwarp();
        if (t < Tn - 2) pair_sync_empty(buf);
        if (act) {
          const Sys<T, T, LAY_PROD, LAY_FULL> sp{sprm, meta_l, tape_b + lane, nullptr, nl, MS};
          const T* x = s_in + buf * W * LANES + lane;
          aba_forward<T, DT, true>(sp, Col<const T>{x, LANES}, Col<const T>{x + nqm * LANES, LANES},
                                   Col<const T>{x + NX * LANES, LANES}, g);
        }
        __threadfence_block();
        __syncwarp();
        pair_arrive_full(buf);
      } else {  // consumer: the adjoint of step t from tape t & 1
        if (act)
          for (int d = 0; d < NX; ++d) cp_async(s_x + d * LANES + lane, ckpt + (t * NX + d) * B + b);
        cp_commit();
        __syncwarp();
        pair_sync_full(buf);
        cp_wait_all();
        if (act) {
          const Sys<T, T, LAY_PROD, LAY_CONS> sc{sprm, meta_l, tape_b + lane, s_adj + lane, nl, MS};
          Col<const T> q{s_x + lane, LANES}, qd{s_x + nqm * LANES + lane, LANES};
          T* gt = gtau + t * nvm * B + b;
          step_adjoint<T, DT>(sc, q, qd, gq, gqd, Col<T>{gt, B}, gm, g, m.dt, m.integ);
          for (int d = nv; d < nvm; ++d) gt[d * B] = T(0);
          if (gtraj) {
            const T* gx = gtraj + t * NX * B + b;
            for (int d = 0; d < nq; ++d) gq[d] += gx[d * B];
            for (int d = 0; d < nv; ++d) gqd[d] += gx[(nqm + d) * B];
          }
        }
        __syncwarp();
        if (t >= 2) pair_arrive_empty(buf);
      }
    }
    if (!consumer) cp_wait_all();
    if (consumer && act) {
      bool ok = true;
      for (int d = 0; d < nq; ++d) ok &= finite_t(gq[d]);
      for (int d = 0; d < nv; ++d) ok &= finite_t(gqd[d]);
      for (int l = 0; l < nl; ++l) ok &= finite_t(gm[l]);
      if (!ok) m.status[b] |= 1;
      for (int d = 0; d < nqm; ++d) gq0[d * B + b] = gq[d];
      for (int d = 0; d < nvm; ++d) gqd0[d * B + b] = gqd[d];
      for (int l = 0; l < nl; ++l) gm_acc[l * B + slot] = gm[l];
    }
    __syncthreads();  // shared memory is reused by the next unit
    if (!m.persistent) break;
    unit = next_unit(m.counter);
  }
}

// ------------------------------------------------------------------ pipelined rollout
// Two warps per 32-system tile for batches of serial revolute chains: the
// inertia warp runs the q-only articulated-inertia recursion of each step
// (chain_inertia) while the bias warp runs the velocity / bias-force pass, then
// follows the inertia warp link by link through the inward pass, then the
// acceleration pass and the integrator (chain_bias_out / chain_bias_in).  Named
// barriers: LINK(l) = 1 + l (the inertia warp arrives when link l's record is
// written, the bias warp waits before reading it) and Q = 15 (the bias warp
// arrives when the state of the next step is in place, the inertia warp waits).
// Per tile both warps execute Q Tn times and every LINK(l), l < the tile's
// longest chain, once per step, whatever their systems; an arrival at LINK(l)
// for step t + 1 follows the Q wait that follows the bias warp's LINK(l) wait of
// step t, and the bias warp's next Q arrival follows LINK waits that follow the
// inertia warp's Q wait.  Chains of up to 14 links.
constexpr int PIPE_MAX_LINKS = 14;
__device__ __forceinline__ void bar_sync_id(int id) { asm volatile("bar.sync %0, 64;\n" ::"r"(id) : "memory"); }
__device__ __forceinline__ void bar_arrive_id(int id) { asm volatile("bar.arrive %0, 64;\n" ::"r"(id) : "memory"); }

__host__ __device__ __forceinline__ long long pipe_fwd_smem_per_tile(int maxL, int nx, int nv) {
  return (long long)maxL * (NPRM + 1 + EX_N + BS_N) + nx + 2LL * nv;
}

template <class T, class DT>
__global__ void __launch_bounds__(2 * LANES, 1)
k_rollout_pipe(DevModel<T> m, const T* __restrict__ q0, const T* __restrict__ qd0, const T* __restrict__ tau,
               long long Tn, int k, T* ckpt, T* qT, T* qdT, T* traj) {
  const int warp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const bool bias = warp == 0;
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const long long L = m.maxL;
  const V3<T> g{m.g0, m.g1, m.g2};
  constexpr int MS = (int)(sizeof(T) / sizeof(int));
  constexpr int BAR_Q = 15;
  T* s_prm = reinterpret_cast<T*>(g_smem);
  T* s_meta = s_prm + L * NPRM * LANES;
  T* s_ex = s_meta + L * LANES;
  T* s_bs = s_ex + L * EX_N * LANES;
  T* s_state = s_bs + L * BS_N * LANES;
  T* s_tau = s_state + (long long)NX * LANES;  // [2][nvm][LANES]
  int* meta_l = reinterpret_cast<int*>(s_meta + lane);
  int unit = m.persistent ? next_unit(m.counter) : (int)blockIdx.x;
  while ((long long)unit * LANES < B) {
    const int slot = unit * LANES + lane;
    const bool act = slot < B;
    const int b = act ? m.sys_of_slot[slot] : 0;
    const int nl = act ? m.nl[slot] : 0;
    const int links = m.nl[unit * LANES];  // slots are sorted by link count: the tile's longest
    if (bias && act) {
      const T* gprm = m.prm + (long long)unit * L * NPRM * LANES + lane;
      const int* gmeta = m.meta + (long long)unit * L * LANES + lane;
      for (int l = 0; l < nl; ++l) {
        for (int f = 0; f < NPRM; ++f) s_prm[(l * NPRM + f) * LANES + lane] = gprm[(l * NPRM + f) * LANES];
        meta_l[l * LANES * MS] = gmeta[l * LANES];
      }
    }
    __syncthreads();
    const Sys<T> s{s_prm + lane, meta_l, nullptr, nullptr, nl, MS};
    Col<T> q{s_state + lane, LANES}, qd{s_state + nqm * LANES + lane, LANES};
    T* ex = s_ex + lane;
    T* bs = s_bs + lane;
    if (bias) {
      if (act) {
        if (Tn > 0)
          for (int d = 0; d < nvm; ++d) cp_async(s_tau + d * LANES + lane, tau + (long long)d * B + b);
        for (int d = 0; d < nqm; ++d) q[d] = q0[d * B + b];
        for (int d = 0; d < nvm; ++d) qd[d] = qd0[d * B + b];
        if (traj) {
          for (int d = 0; d < nqm; ++d) traj[d * B + b] = q[d];
          for (int d = 0; d < nvm; ++d) traj[(nqm + d) * B + b] = qd[d];
        }
      }
      cp_commit();
      __threadfence_block();
      __syncwarp();
      if (Tn > 0) bar_arrive_id(BAR_Q);
    }
    for (long long t = 0; t < Tn; ++t) {
      if (!bias) {  // inertia warp
        __syncwarp();
        bar_sync_id(BAR_Q);
        chain_inertia<T, DT>(s, Col<const T>{q.p, LANES}, ex,
                             [&](int l) {
                               __threadfence_block();
                               __syncwarp();
                               bar_arrive_id(1 + l);
                             },
                             links);
      } else {  // bias warp
        if (act && ckpt && t % k == 0) {
          T* c = ckpt + (t / k) * NX * B + b;
          for (int d = 0; d < nqm; ++d) c[d * B] = q[d];
          for (int d = 0; d < nvm; ++d) c[(nqm + d) * B] = qd[d];
        }
        if (act && t + 1 < Tn) {
          T* nb = s_tau + ((t + 1) & 1) * nvm * LANES + lane;
          for (int d = 0; d < nvm; ++d) cp_async(nb + d * LANES, tau + ((t + 1) * nvm + d) * B + b);
        }
        cp_commit();
        cp_wait_all_but_newest();
        if (act) chain_bias_out(s, Col<const T>{q.p, LANES}, Col<const T>{qd.p, LANES}, bs);
        chain_bias_in<T, DT>(s, q, qd, Col<const T>{s_tau + (t & 1) * nvm * LANES + lane, LANES}, g, ex, bs,
                             [&](int l) {
                               __syncwarp();
                               bar_sync_id(1 + l);
                             },
                             links, m.dt, m.integ);
        if (act && traj) {
          T* c = traj + (t + 1) * NX * B + b;
          for (int d = 0; d < nqm; ++d) c[d * B] = q[d];
          for (int d = 0; d < nvm; ++d) c[(nqm + d) * B] = qd[d];
        }
        __threadfence_block();
        __syncwarp();
        if (t + 1 < Tn) bar_arrive_id(BAR_Q);
      }
    }
    if (bias) {
      cp_wait_all();
      if (act) {
        bool ok = true;
        for (int d = 0; d < nqm; ++d) ok &= finite_t(q[d]);
        for (int d = 0; d < nvm; ++d) ok &= finite_t(qd[d]);
        if (!ok) m.status[b] |= 1;
        for (int d = 0; d < nqm; ++d) qT[d * B + b] = q[d];
        for (int d = 0; d < nvm; ++d) qdT[d * B + b] = qd[d];
      }
    }
    __syncthreads();  // shared memory is reused by the next unit
    if (!m.persistent) break;
    unit = next_unit(m.counter);
  }
}

}  // namespace host
}  // namespace abasim

#include "wpipe.cuh"

namespace abasim {
namespace host {

template <class T>
using BackwardKernel = void (*)(DevModel<T>, const T*, const T*, long long, int, const T*, const T*, const T*,
                                T*, T*, T*, T*, T*);

template <class T>
using RolloutKernel = void (*)(DevModel<T>, const T*, const T*, const T*, long long, int, T*, T*, T*, T*);

// Declared here; defined and explicitly instantiated only in the unit of each
// storage mode, so that the three adjoint-kernel variants compile in parallel.
template <class T, class DT, int ST>
BackwardKernel<T> backward_kernel();
// The contact-model kernels (global storage), instantiated in their own units.
template <class T, class DT>
RolloutKernel<T> rollout_contact_kernel();
template <class T, class DT>
BackwardKernel<T> backward_contact_kernel();
template <class T, class DT>
BackwardKernel<T> backward_pipe_kernel();
// The world-aligned kernels (tape on chip or in global memory), instantiated in
// their own units.
template <class T, class DT>
RolloutKernel<T> wrollout_kernel(bool onchip);
template <class T, class DT>
BackwardKernel<T> wbackward_kernel(bool onchip);
template <class T, class DT>
BackwardKernel<T> wbackward_pipe_kernel(bool onchip);

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


// Grid size and mode of a batched launch; resets the ticket of persistent launches.
// A work unit is one block of `threads` (default h->block) threads covering
// `slots` slots (default: one per thread; the pipelined adjoint runs two warps
// on one 32-slot tile).
template <class K>
int launch_shape(sim_handle* h, K kernel, int* grid, int* persistent, size_t shm, void* stream, int threads = 0,
                 int slots = 0) {
  if (threads == 0) threads = h->block;
  if (slots == 0) slots = threads;
  const int units = (h->B + slots - 1) / slots;
  *grid = units;
  *persistent = 0;
  if (h->schedule != SIM_SCHED_PERSISTENT) return SIM_OK;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, shm);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
  const int cap = std::max(1, per_sm) * std::max(1, h->sms);
  *grid = std::min(units, cap);
  *persistent = 1;
  e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), S(stream));
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "work ticket reset");
}

// Storage mode and dynamic shared memory of a launch: the most on-chip mode that
// fits the per-block opt-in limit and (in auto mode) adds no wave of blocks over
// the all-global kernel.
template <class T, class K0, class K1, class K2>
int choose_storage(sim_handle* h, K0 k_global, K1 k_hybrid, K2 k_smem, bool bwd, int* st, size_t* bytes) {
  *st = ST_GLOBAL;
  *bytes = 0;
  if (h->tape_space == SIM_TAPE_GLOBAL || sizeof(T) != 4) return SIM_OK;
  int limit = 0;
  cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
  int per_sm_g = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_g, k_global, h->block, 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
  const long long units = (h->B + h->block - 1) / h->block;
  const long long sms = std::max(1, h->sms);
  auto waves = [&](int per_sm) { return per_sm > 0 ? (units + sms * per_sm - 1) / (sms * per_sm) : 1LL << 40; };
  const int modes[2] = {ST_SMEM, ST_HYBRID};
  for (int mode : modes) {
    const size_t need = (size_t)(h->block / LANES) *
                        smem_per_tile(h->maxL, h->nq_max + h->nv_max, h->nv_max, bwd, mode) * LANES * sizeof(T);
    if (need > (size_t)limit) continue;
    const void* kern = mode == ST_SMEM ? (const void*)k_smem : (const void*)k_hybrid;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, h->block, need);
    if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
    const bool automatic = h->tape_space == SIM_TAPE_AUTO || h->tape_space == SIM_TAPE_ONE_WARP;
    if (automatic && waves(per_sm) > waves(per_sm_g)) continue;
    if (h->tape_space == SIM_TAPE_SHARED && mode != ST_SMEM) break;
    *st = mode;
    *bytes = need;
    return SIM_OK;
  }
  if (h->tape_space == SIM_TAPE_SHARED) return fail(h, SIM_EUNSUPPORTED, "tape does not fit in shared memory");
  return SIM_OK;
}

// Shared-memory carve-out (percent of the SM's maximum) that holds every block an
// SM must run at once for a single wave of `slots_per_block`-system units, plus one,
// each needing `bytes`: the rest of the SM's unified storage stays L1.
inline int l1_carveout(const sim_handle* h, int slots_per_block, size_t bytes) {
  const long long units = (h->B + slots_per_block - 1) / slots_per_block;
  const long long sms = std::max(1, h->sms);
  const long long per_sm = (units + sms - 1) / sms + 1;
  int sm_smem = 0;
  if (cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device) != cudaSuccess ||
      sm_smem <= 0)
    return 100;
  const long long want = per_sm * ((long long)bytes + 1024);
  return (int)std::min(100LL, std::max(1LL, (100 * want + sm_smem - 1) / sm_smem));
}

// Storage of a world-aligned launch: the tape on chip when a block's tiles fit the
// per-block opt-in limit and that adds no wave of blocks over the global-tape
// kernel (whose blocks still keep their state and input streams on chip).
template <class T, class K>
int choose_w(sim_handle* h, K k_on, K k_off, bool bwd, bool* onchip, size_t* bytes) {
  int limit = 0;
  cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
  const int tiles = h->block / LANES;
  const int nx = h->nq_max + h->nv_max;
  const size_t need_on = (size_t)tiles * w_smem_per_tile(h->maxL, nx, h->nv_max, bwd, true, h->wdepth * WSW) * LANES * sizeof(T);
  const size_t need_off = (size_t)tiles * w_smem_per_tile(h->maxL, nx, h->nv_max, bwd, false, 0) * LANES * sizeof(T);
  if (need_off > (size_t)limit) return fail(h, SIM_EUNSUPPORTED, "the working state does not fit in shared memory");
  e = cudaFuncSetAttribute((const void*)k_off, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_off);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
  // the global-tape kernel: shared memory for the blocks an SM holds at once, the rest of the SM's
  // unified L1 / shared storage as L1 for the tape lines the passes prefetch
  e = cudaFuncSetAttribute((const void*)k_off, cudaFuncAttributePreferredSharedMemoryCarveout,
                           l1_carveout(h, h->block, need_off));
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory carve-out");
  *onchip = false;
  *bytes = need_off;
  if (need_on > (size_t)limit) return SIM_OK;
  e = cudaFuncSetAttribute((const void*)k_on, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_on);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
  int per_on = 0, per_off = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_on, k_on, h->block, need_on);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_off, k_off, h->block, need_off);
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
  const long long units = (h->B + h->block - 1) / h->block;
  const long long sms = std::max(1, h->sms);
  auto waves = [&](int per_sm) { return per_sm > 0 ? (units + sms * per_sm - 1) / (sms * per_sm) : 1LL << 40; };
  if (waves(per_on) <= waves(per_off)) {
    *onchip = true;
    *bytes = need_on;
  }
  return SIM_OK;
}

// The world-aligned path applies to models of revolute joints without contact
// spheres or limits whose state and input streams fit a block's shared memory,
// under SIM_TAPE_ALIGNED, or under SIM_TAPE_AUTO unless the link-frame two-warp
// kernels apply and run faster: the pipelined rollout of serial chains short
// enough for its on-chip tapes, and the link-frame pipelined adjoint of such
// chains when the world-aligned one's two tapes do not fit a block or the
// pivots are FP64 (7-DOF chains, FP32, per 1000-step rollout: world-aligned
// adjoint 10.8 ms against 13.1; with FP64 pivots 40.3 against 34.5).
template <class T, class DT>
bool use_aligned(const sim_handle* h, bool rollout, int k) {
  if (!h->all_revolute || (rollout && h->state64)) return false;
  if (h->tape_space != SIM_TAPE_AUTO && h->tape_space != SIM_TAPE_ALIGNED &&
      h->tape_space != SIM_TAPE_ALIGNED_PIPELINED)
    return false;
  int limit = 0;
  if (cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) return false;
  const int nx = h->nq_max + h->nv_max;
  const size_t streams = (size_t)(h->block / LANES) * w_smem_per_tile(h->maxL, nx, h->nv_max, !rollout, false, 0) * LANES *
                         sizeof(T);
  if (streams > (size_t)limit) return false;
  if (h->tape_space != SIM_TAPE_AUTO || !h->all_chains) return true;
  if (rollout) return !(h->maxL <= PIPE_MAX_LINKS);
  const bool link_pipe = sizeof(T) == 4 && k == 1 &&
                         (size_t)pipe_smem_per_tile(h->maxL, nx, h->nv_max) * LANES * sizeof(T) <= (size_t)limit;
  if (!link_pipe) return true;
  return sizeof(DT) == sizeof(T) &&
         (size_t)wpipe_smem_per_tile(h->maxL, nx, h->nv_max, true, h->wdepth * WSW) * LANES * sizeof(T) <= (size_t)limit;
}

template <class T, class DT>
int launch_wrollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T_, int k, void* ckpt,
                    void* qT, void* qdT, void* traj, void* stream) {
  DevModel<T> m = dev_model<T>(h);
  const RolloutKernel<T> k_on = wrollout_kernel<T, DT>(true), k_off = wrollout_kernel<T, DT>(false);
  bool onchip = false;
  size_t shm = 0;
  int rc = choose_w<T>(h, k_on, k_off, false, &onchip, &shm);
  if (rc != SIM_OK) return rc;
  const RolloutKernel<T> kern = onchip ? k_on : k_off;
  h->last_storage = onchip ? 4 : 5;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream);
  if (rc != SIM_OK) return rc;
  kern<<<grid, h->block, shm, S(stream)>>>(m, (const T*)q0, (const T*)qd0, (const T*)tau, (long long)T_, k,
                                           (T*)ckpt, (T*)qT, (T*)qdT, (T*)traj);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "rollout launch");
}

// The pipelined world-aligned adjoint (two warps per 32-system tile, k = 1):
// tapes on chip when one tile's fit a block, else in global memory.
template <class T, class DT>
int launch_wbackward_pipe(sim_handle* h, const void* ckpt, const void* tau, int64_t T_, const void* gqT,
                          const void* gqdT, const void* gtraj, void* gq0, void* gqd0, void* gtau, void* gmass,
                          void* stream) {
  DevModel<T> m = dev_model<T>(h);
  int limit = 0;
  cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
  const int nx = h->nq_max + h->nv_max;
  const size_t need_on = (size_t)wpipe_smem_per_tile(h->maxL, nx, h->nv_max, true, h->wdepth * WSW) * LANES * sizeof(T);
  const size_t need_off = (size_t)wpipe_smem_per_tile(h->maxL, nx, h->nv_max, false, 0) * LANES * sizeof(T);
  const bool onchip = need_on <= (size_t)limit;
  if (!onchip && !h->wtape2) return fail(h, SIM_EUNSUPPORTED, "no second tape for the pipelined adjoint");
  const size_t shm = onchip ? need_on : need_off;
  const BackwardKernel<T> kern = wbackward_pipe_kernel<T, DT>(onchip);
  e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
  if (!onchip) {  // shared memory for the blocks an SM holds at once, the rest of the SM's storage as L1
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             l1_carveout(h, LANES, shm));
    if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory carve-out");
  }
  h->last_storage_bwd = onchip ? 6 : 7;
  int grid = 0;
  int rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream, 2 * LANES, LANES);
  if (rc != SIM_OK) return rc;
  kern<<<grid, 2 * LANES, shm, S(stream)>>>(m, (const T*)ckpt, (const T*)tau, (long long)T_, 1, (const T*)gqT,
                                            (const T*)gqdT, (const T*)gtraj, (T*)gq0, (T*)gqd0, (T*)gtau,
                                            (T*)h->gm_acc, (T*)h->wtape2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
  if (gmass) {
    k_gather_mass_grad<T><<<(h->L_total + 255) / 256, 256, 0, S(stream)>>>((const T*)h->gm_acc, h->link_slot,
                                                                          h->L_total, (T*)gmass);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "mass-gradient launch");
  }
  return SIM_OK;
}

template <class T, class DT>
int launch_wbackward(sim_handle* h, const void* ckpt, const void* tau, int64_t T_, int k, const void* gqT,
                     const void* gqdT, const void* gtraj, void* gq0, void* gqd0, void* gtau, void* gmass, void* work,
                     void* stream) {
  DevModel<T> m = dev_model<T>(h);
  if (k == 1 && T_ > 0 && h->tape_space != SIM_TAPE_ALIGNED)
    return launch_wbackward_pipe<T, DT>(h, ckpt, tau, T_, gqT, gqdT, gtraj, gq0, gqd0, gtau, gmass, stream);
  const BackwardKernel<T> k_on = wbackward_kernel<T, DT>(true), k_off = wbackward_kernel<T, DT>(false);
  bool onchip = false;
  size_t shm = 0;
  int rc = choose_w<T>(h, k_on, k_off, true, &onchip, &shm);
  if (rc != SIM_OK) return rc;
  const BackwardKernel<T> kern = onchip ? k_on : k_off;
  h->last_storage_bwd = onchip ? 4 : 5;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream);
  if (rc != SIM_OK) return rc;
  kern<<<grid, h->block, shm, S(stream)>>>(m, (const T*)ckpt, (const T*)tau, (long long)T_, k, (const T*)gqT,
                                           (const T*)gqdT, (const T*)gtraj, (T*)gq0, (T*)gqd0, (T*)gtau,
                                           (T*)h->gm_acc, (T*)work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "backward launch");
  if (gmass) {
    k_gather_mass_grad<T><<<(h->L_total + 255) / 256, 256, 0, S(stream)>>>((const T*)h->gm_acc, h->link_slot,
                                                                          h->L_total, (T*)gmass);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "mass-gradient launch");
  }
  return SIM_OK;
}

template <class T, class DT>
int launch_rollout(sim_handle* h, const void* q0, const void* qd0, const void* tau, int64_t T_,
                   int k, void* ckpt, void* qT, void* qdT, void* traj, void* stream) {
  if (use_aligned<T, DT>(h, true, k)) return launch_wrollout<T, DT>(h, q0, qd0, tau, T_, k, ckpt, qT, qdT, traj, stream);
  if (h->tape_space == SIM_TAPE_ALIGNED || h->tape_space == SIM_TAPE_ALIGNED_PIPELINED)
    return fail(h, SIM_EUNSUPPORTED,
                "the world-aligned kernels need revolute joints only, no contact spheres or limits, FP32 state sums "
                "and a state that fits a block's shared memory");
  DevModel<T> m = dev_model<T>(h);
  size_t shm = 0;
  int st = ST_GLOBAL;
  int rc = SIM_OK;
  RolloutKernel<T> kern = k_rollout<T, DT, ST_GLOBAL>;
  int threads = h->block;
  if (h->ctape) {
    kern = rollout_contact_kernel<T, DT>();
  } else {
    bool piped = false;  // the pipelined rollout, any precision
    if (h->all_chains && h->maxL <= PIPE_MAX_LINKS && !h->state64 &&
        (h->tape_space == SIM_TAPE_AUTO || h->tape_space == SIM_TAPE_PIPELINED)) {
      const size_t need =
          (size_t)pipe_fwd_smem_per_tile(h->maxL, h->nq_max + h->nv_max, h->nv_max) * LANES * sizeof(T);
      int limit = 0;
      cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
      if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
      if (need <= (size_t)limit) {
        kern = k_rollout_pipe<T, DT>;
        e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
        st = ST_PIPE;
        shm = need;
        threads = 2 * LANES;
        piped = true;
      }
    }
    if (!piped && h->tape_space == SIM_TAPE_PIPELINED)
      return fail(h, SIM_EUNSUPPORTED,
                  "the pipelined rollout needs serial revolute chains of at most 14 links and FP32 state accumulation");
    if constexpr (sizeof(T) == 4) {  // the other on-chip modes: FP32 storage only
      if (!piped) {
        rc = choose_storage<T>(h, k_rollout<T, DT, ST_GLOBAL>, k_rollout<T, DT, ST_HYBRID>,
                               k_rollout<T, DT, ST_SMEM>, false, &st, &shm);
        if (st == ST_SMEM) kern = k_rollout<T, DT, ST_SMEM>;
        if (st == ST_HYBRID) kern = k_rollout<T, DT, ST_HYBRID>;
      }
    }
  }
  if (rc != SIM_OK) return rc;
  h->last_storage = st;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream, threads, st == ST_PIPE ? LANES : threads);
  if (rc != SIM_OK) return rc;
  kern<<<grid, threads, shm, S(stream)>>>(m, (const T*)q0, (const T*)qd0, (const T*)tau, (long long)T_,
                                           k, (T*)ckpt, (T*)qT, (T*)qdT, (T*)traj);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "rollout launch");
}

template <class T, class DT>
int launch_backward(sim_handle* h, const void* ckpt, const void* tau, int64_t T_, int k,
                    const void* gqT, const void* gqdT, const void* gtraj, void* gq0, void* gqd0,
                    void* gtau, void* gmass, void* work, void* stream) {
  if (use_aligned<T, DT>(h, false, k))
    return launch_wbackward<T, DT>(h, ckpt, tau, T_, k, gqT, gqdT, gtraj, gq0, gqd0, gtau, gmass, work, stream);
  if (h->tape_space == SIM_TAPE_ALIGNED || h->tape_space == SIM_TAPE_ALIGNED_PIPELINED)
    return fail(h, SIM_EUNSUPPORTED, "the world-aligned kernels need revolute joints only, no contact spheres or "
                                     "limits, and a state that fits a block's shared memory");
  DevModel<T> m = dev_model<T>(h);
  size_t shm = 0;
  int st = ST_GLOBAL;
  int rc = SIM_OK;
  BackwardKernel<T> kern = backward_kernel<T, DT, ST_GLOBAL>();
  int threads = h->block;
  if (h->ctape) {
    kern = backward_contact_kernel<T, DT>();
  } else if constexpr (sizeof(T) == 4) {  // on-chip modes: FP32 storage only
    bool piped = false;
    if (k == 1 && T_ > 0 && h->all_chains &&
        (h->tape_space == SIM_TAPE_AUTO || h->tape_space == SIM_TAPE_PIPELINED)) {
      // the pipelined two-warp adjoint, when its shared memory fits one block
      int limit = 0;
      cudaError_t e = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
      if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory limit query");
      const size_t need =
          (size_t)pipe_smem_per_tile(h->maxL, h->nq_max + h->nv_max, h->nv_max) * LANES * sizeof(T);
      if (need <= (size_t)limit) {
        kern = backward_pipe_kernel<T, DT>();
        e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        if (e != cudaSuccess) return cuda_fail(h, e, "shared-memory opt-in");
        st = ST_PIPE;
        shm = need;
        threads = 2 * LANES;
        piped = true;
      }
    }
    if (!piped && h->tape_space == SIM_TAPE_PIPELINED)
      return fail(h, SIM_EUNSUPPORTED,
                  "the pipelined adjoint needs k = 1, serial revolute chains and a tile that fits in shared memory");
    if (!piped) {
      const BackwardKernel<T> k_hyb = backward_kernel<T, DT, ST_HYBRID>();
      const BackwardKernel<T> k_smem = backward_kernel<T, DT, ST_SMEM>();
      rc = choose_storage<T>(h, kern, k_hyb, k_smem, true, &st, &shm);
      if (st == ST_SMEM) kern = k_smem;
      if (st == ST_HYBRID) kern = k_hyb;
    }
  }
  if (rc != SIM_OK) return rc;
  h->last_storage_bwd = st;
  int grid = 0;
  rc = launch_shape(h, kern, &grid, &m.persistent, shm, stream, threads, st == ST_PIPE ? LANES : threads);
  if (rc != SIM_OK) return rc;
  kern<<<grid, threads, shm, S(stream)>>>(m, (const T*)ckpt, (const T*)tau, (long long)T_, k,
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


// One step with the per-link tape at `tape`.
template <class T, class DT>
int launch_step_with_tape(sim_handle* h, const void* q, const void* qd, const void* tau, void* q_out,
                          void* qd_out, void* tape, void* stream) {
  DevModel<T> m = dev_model<T>(h);
  m.tape = (T*)tape;
  const int grid = (h->B + h->block - 1) / h->block;
  const RolloutKernel<T> kern = h->ctape ? rollout_contact_kernel<T, DT>() : k_rollout<T, DT, ST_GLOBAL>;
  kern<<<grid, h->block, 0, S(stream)>>>(m, (const T*)q, (const T*)qd, (const T*)tau, 1LL, 1, (T*)nullptr,
                                         (T*)q_out, (T*)qd_out, (T*)nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "step launch");
}

template <class T>
int launch_jvp(sim_handle* h, const void* q, const void* qd, const void* tau, const void* dq,
               const void* dqd, const void* dtau, void* q_out, void* qd_out, void* dq_out,
               void* dqd_out, void* work, void* stream) {
  const int grid = (h->B + h->block - 1) / h->block;
  k_step_jvp<T, T><<<grid, h->block, 0, S(stream)>>>(
      dev_model<T>(h), (const T*)q, (const T*)qd, (const T*)tau, (const T*)dq, (const T*)dqd,
      (const T*)dtau, (T*)q_out, (T*)qd_out, (T*)dq_out, (T*)dqd_out, (Dual<T>*)work);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "jvp launch");
}

template <class T>
int launch_set_masses(sim_handle* h, const void* mass, void* stream) {
  const int grid = (h->L_total + 255) / 256;
  k_set_masses<T><<<grid, 256, 0, S(stream)>>>((T*)h->prm, h->link_slot, h->L_total, h->B, h->maxL,
                                              (const T*)mass);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : cuda_fail(h, e, "set_masses launch");
}

}  // namespace host
}  // namespace abasim
