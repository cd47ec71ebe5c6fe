// The pipelined adjoint of the world-aligned step: two warps per 32-system tile,
// for revolute models without contacts or limits and a checkpoint every step.
// With every step's initial state checkpointed, the recompute of step t (Sec. 3.2,
// Eq. 7: Z^t = G(x^t)) does not depend on the adjoint of step t + 1, so a producer
// warp recomputes step t into one of two tapes while a consumer warp runs the
// adjoint of step t + 1 from the other.  The hand-off is the named-barrier
// protocol of the link-frame pipelined adjoint: FULL(b) (the producer arrives when
// tape b holds its step; the consumer waits) and EMPTY(b) (the consumer arrives
// when it has finished a step from tape b that the producer will reuse; the
// producer waits before overwriting).  Both warps execute every barrier the same
// number of times whatever their systems, and neither arrives twice at a barrier
// before the other's matching wait.  The tapes, the adjoint record, the model
// constants and the inputs live on chip when the block's shared memory holds them
// (ONCHIP), else in global memory (the second tape in the handle's extra scratch)
// with their lines prefetched.
#pragma once

namespace abasim {
namespace host {

// Scalars per tile: the state adjoint and per-link mass-gradient sums; with
// ONCHIP also both tapes, the adjoint record, model constants and meta words, the
// two warps' stacks of parent values (sd scalars per system each) and the
// producer's double-buffered inputs (x^t, tau^t).  Without ONCHIP the producer
// reads its inputs from global memory, their lines prefetched a step ahead.
__host__ __device__ __forceinline__ long long wpipe_smem_per_tile(int maxL, int nx, int nv, bool onchip, int sd) {
  const long long state = nx + maxL;
  if (!onchip) return state;
  return (long long)maxL * (2 * NWT + NWA + NPRM_W + 1) + 2LL * sd + state + 2LL * (nx + nv);
}

template <class T, class DT, bool ONCHIP>
__global__ void __launch_bounds__(2 * LANES, 1)
k_wbackward_pipe(DevModel<T> m, const T* __restrict__ ckpt, const T* __restrict__ tau, long long Tn, int k,
                 const T* __restrict__ gqT, const T* __restrict__ gqdT, const T* __restrict__ gtraj, T* gq0,
                 T* gqd0, T* gtau, T* gm_acc, T* tape2) {
  const int warp = threadIdx.x / LANES, lane = threadIdx.x % LANES;
  const bool consumer = warp == 0;
  const long long B = m.B;
  const int nqm = m.nq_max, nvm = m.nv_max, NX = nqm + nvm;
  const long long L = m.maxL;
  const V3<T> g{m.g0, m.g1, m.g2};
  constexpr int MS = (int)(sizeof(T) / sizeof(int));
  T* base = reinterpret_cast<T*>(g_smem);
  T *s_tape = nullptr, *s_adj = nullptr, *s_prm = nullptr, *s_meta = nullptr, *s_in = nullptr;
  T* s_stk = nullptr;
  const long long sdw = (long long)m.wdepth * WSW;  // stack scalars per system
  if (ONCHIP) {
    s_tape = base;  // [2][L][NWT][LANES]
    base += 2 * L * NWT * LANES;
    s_adj = base;
    base += L * NWA * LANES;
    s_prm = base;
    base += L * NPRM_W * LANES;
    s_meta = base;
    base += L * LANES;
    s_stk = base;  // [2][sdw][LANES]: the producer's stack, then the consumer's
    base += 2 * sdw * LANES;
  }
  T* s_state = base;
  T* s_gm = s_state + (long long)NX * LANES;
  if (ONCHIP) s_in = s_gm + L * LANES;  // [2][NX + nvm][LANES]
  const int W = NX + nvm;
  int unit = m.persistent ? next_unit(m.counter) : (int)blockIdx.x;
  while ((long long)unit * LANES < B) {
    const int slot = unit * LANES + lane;
    const bool act = slot < B;
    const int b = act ? m.sys_of_slot[slot] : 0;
    const int nl = act ? m.nl[slot] : 0;
    const int nq = act ? (m.nqv[slot] & 0xffff) : 0, nv = act ? (m.nqv[slot] >> 16) : 0;
    const T* gprm = m.prm + (long long)unit * L * NPRM * LANES + lane;
    const int* gmeta = m.meta + (long long)unit * L * LANES + lane;
    int* meta_l = ONCHIP ? reinterpret_cast<int*>(s_meta + lane) : nullptr;
    if (ONCHIP && consumer && act) {
      for (int l = 0; l < nl; ++l) {
        for (int f = 0; f < NPRM_W; ++f) s_prm[(l * NPRM_W + f) * LANES + lane] = gprm[(l * NPRM + f) * LANES];
        meta_l[l * LANES * MS] = gmeta[l * LANES];
      }
    }
    __syncthreads();
    auto tape_of = [&](int buf) -> T* {
      if (ONCHIP) return s_tape + buf * L * NWT * LANES + lane;
      return (buf ? tape2 : m.tape) + (long long)unit * L * NWT * LANES + lane;
    };
    const int who = consumer ? 1 : 0;  // each warp walks its own stack
    auto sys_of_buf = [&](int buf) -> WSys<T> {
      if (ONCHIP)
        return WSys<T>{s_prm + lane, meta_l, tape_of(buf), s_adj + lane, nl, MS, NPRM_W, 0,
                       s_stk + who * sdw * LANES + lane};
      return WSys<T>{gprm, gmeta, tape_of(buf), m.adj + (long long)unit * L * NWA * LANES + lane, nl, 1, NPRM, m.pf,
                     w_stack(m, who, unit, lane)};
    };
    // the producer's inputs of step t: x^t and tau^t (the system's own coordinates)
    auto fetch = [&](long long t, int buf) {
      T* dst = s_in + buf * W * LANES + lane;
      for (int d = 0; d < nq; ++d) cp_async(dst + d * LANES, ckpt + (t * NX + d) * B + b);
      for (int d = 0; d < nv; ++d) cp_async(dst + (nqm + d) * LANES, ckpt + (t * NX + nqm + d) * B + b);
      for (int d = 0; d < nv; ++d) cp_async(dst + (NX + d) * LANES, tau + (t * nvm + d) * B + b);
    };
    if (ONCHIP && !consumer) {
      if (act && Tn > 0) fetch(Tn - 1, (int)((Tn - 1) & 1));
      cp_commit();
    }
    const Col<T> gq{s_state + lane, LANES}, gqd{s_state + nqm * LANES + lane, LANES}, gm{s_gm + lane, LANES};
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
      if (!consumer) {  // producer: recompute step t into tape t & 1
        if (ONCHIP) {
          if (act && t > 0) fetch(t - 1, (int)((t - 1) & 1));
          cp_commit();
          cp_wait_all_but_newest();
        } else if (act && t > 0 && m.pf > 0) {
          const T* xn = ckpt + (t - 1) * NX * B + b;
          for (int d = 0; d < nq; ++d) pf_line(xn + d * B);
          for (int d = 0; d < nv; ++d) pf_line(xn + (nqm + d) * B);
          for (int d = 0; d < nv; ++d) pf_line(tau + ((t - 1) * nvm + d) * B + b);
        }
        __syncwarp();
        if (t < Tn - 2) pair_sync_empty(buf);
        if (act) {
          const WSys<T> sp = sys_of_buf(buf);
          if (ONCHIP) {
            const T* x = s_in + buf * W * LANES + lane;
            wstep_forward<T, DT, true, false>(sp, Col<const T>{x, LANES}, Col<const T>{x + nqm * LANES, LANES},
                                              Col<const T>{x + NX * LANES, LANES}, g, m.dt, m.integ,
                                              Col<T>{nullptr, 0}, Col<T>{nullptr, 0});
          } else {
            const T* x = ckpt + t * NX * B + b;
            wstep_forward<T, DT, true, false>(sp, Col<const T>{x, B}, Col<const T>{x + nqm * B, B},
                                              Col<const T>{tau + t * nvm * B + b, B}, g, m.dt, m.integ,
                                              Col<T>{nullptr, 0}, Col<T>{nullptr, 0});
          }
        }
        __threadfence_block();
        __syncwarp();
        pair_arrive_full(buf);
      } else {  // consumer: the adjoint of step t from tape t & 1
        __syncwarp();
        pair_sync_full(buf);
        if (act) {
          const WSys<T> sc = sys_of_buf(buf);
          T* gt = gtau + t * nvm * B + b;
          wstep_adjoint<T, DT, !ONCHIP && sizeof(T) == 4>(sc, gq, gqd, Col<T>{gt, B}, gm, m.dt, m.integ);
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
    if (ONCHIP && !consumer) cp_wait_all();
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

}  // namespace host
}  // namespace abasim
