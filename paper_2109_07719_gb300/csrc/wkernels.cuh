// Batched rollout and adjoint kernels of the world-aligned step (wstep.cuh) for
// models whose joints are all revolute and that have no contact spheres or joint
// limits.  Thread i handles slot i (systems sorted by link count, longest first);
// the tape and adjoint record are tile-major, [tile][link][field][lane], in
// shared memory when a block's tiles fit (ONCHIP), else in the handle's global
// scratch with the working state and the prefetched input streams still on chip.
#pragma once

#include "wstep.cuh"

namespace abasim {
namespace host {

// Scalars per 32-system tile a world-aligned kernel keeps in shared memory: the
// working state (x for the rollout, the state adjoint and the per-link
// mass-gradient sums for the backward pass); with ONCHIP also the tape (and, for
// the adjoint, the adjoint record), the model constants and meta words, the stack
// of parent values (sd scalars per system) and a double buffer for the per-step
// inputs (tau, plus x^t for the adjoint) fetched one step ahead.  Without ONCHIP
// the stack is in the handle's global scratch and the inputs are read from global
// memory with their lines prefetched a step ahead, and the small shared-memory
// footprint leaves most of the SM's L1 to the prefetched tape lines (staging the
// inputs on chip instead cost more in L1 than it saved in misses).
__host__ __device__ __forceinline__ long long w_smem_per_tile(int maxL, int nx, int nv, bool bwd, bool onchip,
                                                              int sd) {
  const long long state = nx + (bwd ? maxL : 0);
  if (!onchip) return state;
  return (long long)maxL * (NWT + (bwd ? NWA : 0) + NPRM_W + 1) + sd + state + 2LL * (nv + (bwd ? nx : 0));
}

// Stack `which` (0, or 1 for the second warp of the pipelined adjoint) of a tile's
// system at `lane` in the handle's global scratch (null when no system branches).
template <class T>
__device__ __forceinline__ T* w_stack(const DevModel<T>& m, int which, long long tile, long long lane) {
  if (!m.stk) return nullptr;
  const long long tiles = (m.B + LANES - 1) / LANES;
  return m.stk + ((long long)which * tiles + tile) * m.wdepth * WSW * LANES + lane;
}

struct WTile {
  void* tape;
  void* adj;
  void* prm;
  int* meta;
  void* stk;
  void* state;
  void* gm;
  void* stream;
};

template <class T, bool BWD, bool ONCHIP>
__device__ __forceinline__ WTile w_tile(int maxL, int nx, int nv, int sd, int lane) {
  const int tb = threadIdx.x / LANES;
  const long long L = maxL;
  T* base =
      reinterpret_cast<T*>(g_smem) + (long long)tb * w_smem_per_tile(maxL, nx, nv, BWD, ONCHIP, sd) * LANES + lane;
  WTile t{};
  if (ONCHIP) {
    t.tape = base;
    base += L * NWT * LANES;
    t.adj = base;
    if (BWD) base += L * NWA * LANES;
    t.prm = base;
    base += L * NPRM_W * LANES;
    t.meta = reinterpret_cast<int*>(base);
    base += L * LANES;
    t.stk = base;
    base += (long long)sd * LANES;
  }
  t.state = base;
  base += (long long)nx * LANES;
  t.gm = base;
  if (BWD) base += L * LANES;
  t.stream = base;
  return t;
}

// The system view of a slot: constants, meta words and tape on chip (copied in
// here) or in global memory.
template <class T, bool BWD, bool ONCHIP>
__device__ __forceinline__ WSys<T> wsys_of(const DevModel<T>& m, int slot) {
  const long long tile = slot / LANES, lane = slot % LANES;
  const long long L = m.maxL;
  const T* gprm = m.prm + tile * L * NPRM * LANES + lane;
  const int* gmeta = m.meta + tile * L * LANES + lane;
  const int nl = m.nl[slot];
  if (ONCHIP) {
    const WTile t = w_tile<T, BWD, ONCHIP>(m.maxL, m.nq_max + m.nv_max, m.nv_max, m.wdepth * WSW, (int)lane);
    T* sp = (T*)t.prm;
    constexpr int MS = (int)(sizeof(T) / sizeof(int));
    for (int l = 0; l < nl; ++l) {
      for (int f = 0; f < NPRM_W; ++f) sp[(l * NPRM_W + f) * LANES] = gprm[(l * NPRM + f) * LANES];
      t.meta[l * LANES * MS] = gmeta[l * LANES];
    }
    return WSys<T>{sp, t.meta, (T*)t.tape, (T*)t.adj, nl, MS, NPRM_W, 0, (T*)t.stk};
  }
  return WSys<T>{gprm, gmeta, m.tape + tile * L * NWT * LANES + lane, m.adj + tile * L * NWA * LANES + lane, nl, 1,
                 NPRM, m.pf, w_stack(m, 0, tile, lane)};
}

template <class T, class DT, bool ONCHIP>
__device__ __forceinline__ void wrollout_one(const DevModel<T>& m, int slot, const T* __restrict__ q0,
                                             const T* __restrict__ qd0, const T* __restrict__ tau, long long Tn,
                                             int k, T* ckpt, T* qT, T* qdT, T* traj) {
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const V3<T> g{m.g0, m.g1, m.g2};
  const WSys<T> s = wsys_of<T, false, ONCHIP>(m, slot);
  const WTile st = w_tile<T, false, ONCHIP>(m.maxL, NX, nvm, m.wdepth * WSW, slot % LANES);
  const Col<T> q{(T*)st.state, LANES}, qd{(T*)st.state + nqm * LANES, LANES};
  const int nv = m.nqv[slot] >> 16;
  T* sbuf = (T*)st.stream;  // ONCHIP: [2][nvm][LANES], tau one step ahead
  if (ONCHIP) {
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
    if (ONCHIP) {
      if (t + 1 < Tn) {
        T* nb = sbuf + ((t + 1) & 1) * nvm * LANES;
        for (int d = 0; d < nvm; ++d) cp_async(nb + d * LANES, tau + ((t + 1) * nvm + d) * B + b);
      }
      cp_commit();
      cp_wait_all_but_newest();
      tau_t = Col<const T>{sbuf + (t & 1) * nvm * LANES, LANES};
    } else if (t + 1 < Tn && m.pf > 0) {
      for (int d = 0; d < nv; ++d) pf_line(tau + ((t + 1) * nvm + d) * B + b);
    }
    wstep_forward<T, DT, false, true>(s, Col<const T>{q.p, LANES}, Col<const T>{qd.p, LANES}, tau_t, g, m.dt,
                                      m.integ, q, qd);
    if (traj) {
      T* c = traj + (t + 1) * NX * B + b;
      for (int d = 0; d < nqm; ++d) c[d * B] = q[d];
      for (int d = 0; d < nvm; ++d) c[(nqm + d) * B] = qd[d];
    }
  }
  if (ONCHIP) cp_wait_all();
  bool ok = true;
  for (int d = 0; d < nqm; ++d) ok &= finite_t(q[d]);
  for (int d = 0; d < nvm; ++d) ok &= finite_t(qd[d]);
  if (!ok) m.status[b] |= 1;
  for (int d = 0; d < nqm; ++d) qT[d * B + b] = q[d];
  for (int d = 0; d < nvm; ++d) qdT[d * B + b] = qd[d];
}

template <class T, class DT, bool ONCHIP>
__device__ __forceinline__ void wbackward_one(const DevModel<T>& m, int slot, const T* __restrict__ ckpt,
                                              const T* __restrict__ tau, long long Tn, int k,
                                              const T* __restrict__ gqT, const T* __restrict__ gqdT,
                                              const T* __restrict__ gtraj, T* gq0, T* gqd0, T* gtau, T* gm_acc,
                                              T* ring) {
  const int b = m.sys_of_slot[slot];
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const int nq = m.nqv[slot] & 0xffff, nv = m.nqv[slot] >> 16;
  const V3<T> g{m.g0, m.g1, m.g2};
  const WSys<T> s = wsys_of<T, true, ONCHIP>(m, slot);
  const WTile st = w_tile<T, true, ONCHIP>(m.maxL, NX, nvm, m.wdepth * WSW, slot % LANES);
  const Col<T> gq{(T*)st.state, LANES}, gqd{(T*)st.state + nqm * LANES, LANES}, gm{(T*)st.gm, LANES};
  T* sbuf = (T*)st.stream;  // [2][NX + nvm][LANES]: x^t and tau^t, one step ahead (k = 1)
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
  auto step_back = [&](long long t, Col<const T> q, Col<const T> qd, Col<const T> tau_t) {
    wstep_forward<T, DT, true, false>(s, q, qd, tau_t, g, m.dt, m.integ, Col<T>{nullptr, 0}, Col<T>{nullptr, 0});
    T* gt = gtau + t * nvm * B + b;
    wstep_adjoint<T, DT, !ONCHIP && sizeof(T) == 4>(s, gq, gqd, Col<T>{gt, B}, gm, m.dt, m.integ);
    for (int d = nv; d < nvm; ++d) gt[d * B] = T(0);
    if (gtraj) {
      const T* gx = gtraj + t * NX * B + b;
      for (int d = 0; d < nq; ++d) gq[d] += gx[d * B];
      for (int d = 0; d < nv; ++d) gqd[d] += gx[(nqm + d) * B];
    }
  };
  if (k == 1 && ONCHIP) {
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
      step_back(t, Col<const T>{xb, LANES}, Col<const T>{xb + nqm * LANES, LANES},
                Col<const T>{xb + NX * LANES, LANES});
    }
    cp_wait_all();
  } else if (k == 1) {  // inputs straight from global memory, the previous step's lines prefetched
    for (long long t = Tn - 1; t >= 0; --t) {
      if (t > 0 && m.pf > 0) {
        const T* xn = ckpt + (t - 1) * NX * B + b;
        for (int d = 0; d < nq; ++d) pf_line(xn + d * B);
        for (int d = 0; d < nv; ++d) pf_line(xn + (nqm + d) * B);
        for (int d = 0; d < nv; ++d) pf_line(tau + ((t - 1) * nvm + d) * B + b);
      }
      const T* x = ckpt + t * NX * B + b;
      step_back(t, Col<const T>{x, B}, Col<const T>{x + nqm * B, B}, Col<const T>{tau + t * nvm * B + b, B});
    }
  } else {
    const long long nseg = (Tn + k - 1) / k;
    for (long long seg = nseg - 1; seg >= 0; --seg) {
      const long long t0 = seg * k;
      const long long t1 = (t0 + k < Tn) ? t0 + k : Tn;
      const T* xs = ckpt + seg * NX * B + b;
      if (!m.quadratic) {  // replay the segment once, keeping its states (ring by slot)
        T* r0 = ring + slot;
        for (int d = 0; d < NX; ++d) r0[d * B] = xs[d * B];
        for (long long j = 1; j < t1 - t0; ++j) {
          const T* prev = ring + (j - 1) * NX * B + slot;
          T* cur = ring + j * NX * B + slot;
          wstep_forward<T, DT, false, true>(s, Col<const T>{prev, B}, Col<const T>{prev + nqm * B, B},
                                            Col<const T>{tau + (t0 + j - 1) * nvm * B + b, B}, g, m.dt, m.integ,
                                            Col<T>{cur, B}, Col<T>{cur + nqm * B, B});
        }
      }
      for (long long t = t1 - 1; t >= t0; --t) {
        const T* x = ring + (t - t0) * NX * B + slot;
        if (m.quadratic) {  // recompute x^t from the segment checkpoint: t - t0 steps
          T* cur = ring + slot;
          x = t == t0 ? xs : cur;
          if (t > t0) {
            wstep_forward<T, DT, false, true>(s, Col<const T>{xs, B}, Col<const T>{xs + nqm * B, B},
                                              Col<const T>{tau + t0 * nvm * B + b, B}, g, m.dt, m.integ,
                                              Col<T>{cur, B}, Col<T>{cur + nqm * B, B});
            for (long long j = t0 + 1; j < t; ++j)
              wstep_forward<T, DT, false, true>(s, Col<const T>{cur, B}, Col<const T>{cur + nqm * B, B},
                                                Col<const T>{tau + j * nvm * B + b, B}, g, m.dt, m.integ,
                                                Col<T>{cur, B}, Col<T>{cur + nqm * B, B});
          }
        }
        step_back(t, Col<const T>{x, B}, Col<const T>{x + nqm * B, B}, Col<const T>{tau + t * nvm * B + b, B});
      }
    }
  }
  bool ok = true;
  for (int d = 0; d < nq; ++d) ok &= finite_t(gq[d]);
  for (int d = 0; d < nv; ++d) ok &= finite_t(gqd[d]);
  for (int l = 0; l < s.nl; ++l) ok &= finite_t(gm[l]);
  if (!ok) m.status[b] |= 1;
  for (int d = 0; d < nqm; ++d) gq0[d * B + b] = gq[d];
  for (int d = 0; d < nvm; ++d) gqd0[d * B + b] = gqd[d];
  for (int l = 0; l < s.nl; ++l) gm_acc[l * B + slot] = gm[l];
}

template <class T, class DT, bool ONCHIP>
__global__ void k_wrollout(DevModel<T> m, const T* __restrict__ q0, const T* __restrict__ qd0,
                           const T* __restrict__ tau, long long Tn, int k, T* ckpt, T* qT, T* qdT, T* traj) {
  ABASIM_FOR_EACH_SLOT(m, wrollout_one<T, DT, ONCHIP>(m, slot, q0, qd0, tau, Tn, k, ckpt, qT, qdT, traj))
}

template <class T, class DT, bool ONCHIP>
__global__ void k_wbackward(DevModel<T> m, const T* __restrict__ ckpt, const T* __restrict__ tau, long long Tn,
                            int k, const T* __restrict__ gqT, const T* __restrict__ gqdT,
                            const T* __restrict__ gtraj, T* gq0, T* gqd0, T* gtau, T* gm_acc, T* ring) {
  ABASIM_FOR_EACH_SLOT(m, wbackward_one<T, DT, ONCHIP>(m, slot, ckpt, tau, Tn, k, gqT, gqdT, gtraj, gq0, gqd0,
                                                       gtau, gm_acc, ring))
}

}  // namespace host
}  // namespace abasim
