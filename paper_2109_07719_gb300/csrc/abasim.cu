// C-ABI implementation, host side: model validation and packing, handle
// lifetime, argument checks, the static scratch of sim_step_batch_static, and
// dispatch to the per-precision launch functions (kernels.cuh, inst_*.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "contact.cuh"
#include "handle.h"
#include "tree_order.h"
#include "wstep.cuh"

using namespace abasim;
using namespace abasim::host;

namespace {

constexpr int kMaxLinks = 255;
constexpr int kMaxCoords = 1023;

thread_local std::string g_create_error;

}  // namespace

namespace abasim {
namespace host {

int fail(sim_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(sim_handle* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace host
}  // namespace abasim

namespace {

bool is_fp64(const sim_handle* h) { return h->precision == SIM_FP64; }

// ------------------------------------------------------------------ validation

bool near(double a, double b, double tol) { return std::fabs(a - b) <= tol; }

// ------------------------------------------------------------------ joint frames
// The kernels take every revolute joint about its link's z axis.  Each revolute
// link is re-expressed in the frame x' = R x with R a = e_z (a the model's
// axis); a free link keeps its frame.  Row-major 3x3 helpers, double precision.
using M9 = std::array<double, 9>;

M9 mat_mul(const M9& a, const M9& b) {
  M9 o{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
  return o;
}
M9 mat_T(const M9& a) { return M9{a[0], a[3], a[6], a[1], a[4], a[7], a[2], a[5], a[8]}; }
void mat_vec(const M9& a, const double* x, double* y) {
  for (int i = 0; i < 3; ++i) y[i] = a[3 * i] * x[0] + a[3 * i + 1] * x[1] + a[3 * i + 2] * x[2];
}

// A rotation R with R n = e_z for the unit vector n = a / |a|: Rodrigues' rotation
// about n x e_z, R = 1 + K + K^2 / (1 + n.z) with K = skew(n x e_z).  For n.z < 0
// n is first turned by pi about x (diag(1, -1, -1)), which keeps 1 + n.z away from 0.
M9 rotation_to_z(const double* a) {
  const double len = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double n[3] = {a[0] / len, a[1] / len, a[2] / len};
  const bool flip = n[2] < 0;
  if (flip) {
    n[1] = -n[1];
    n[2] = -n[2];
  }
  const double vx = n[1], vy = -n[0];  // n x e_z = (n.y, -n.x, 0)
  const double k = 1.0 / (1.0 + n[2]);
  const M9 K{0, 0, vy, 0, 0, -vx, -vy, vx, 0};
  const M9 K2 = mat_mul(K, K);
  M9 R{};
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + K[i] + k * K2[i];
  return flip ? mat_mul(R, M9{1, 0, 0, 0, -1, 0, 0, 0, -1}) : R;
}

int validate(const sim_model_desc* d, std::string& why) {
  auto bad = [&](const std::string& s) { why = s; return SIM_EINVAL; };
  if (!d) return bad("null model description");
  if (d->n_systems < 1) return bad("n_systems must be >= 1");
  if (d->precision < SIM_FP64 || d->precision > SIM_FP32_D64) return bad("unknown precision");
  if (d->integrator != SIM_SEMI_IMPLICIT_EULER && d->integrator != SIM_EXPLICIT_EULER)
    return bad("unknown integrator");
  if (d->flags & ~SIM_KEEP_SYSTEM_ORDER) return bad("unknown flag bits");
  if (!(d->dt > 0) || !std::isfinite(d->dt)) return bad("dt must be finite and > 0");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(d->gravity[i])) return bad("gravity must be finite");
  if (!d->sys_link_offset || !d->parent || !d->joint_type || !d->axis || !d->X_tree || !d->mass ||
      !d->com || !d->I_com)
    return bad("null model array");
  if (d->sys_link_offset[0] != 0) return bad("sys_link_offset[0] must be 0");
  bool any_contact = false;
  for (int b = 0; b < d->n_systems; ++b) {
    const int o0 = d->sys_link_offset[b], o1 = d->sys_link_offset[b + 1];
    const int n = o1 - o0;
    char buf[160];
    if (n < 1 || n > kMaxLinks) {
      snprintf(buf, sizeof buf, "system %d has %d links (1..%d allowed)", b, n, kMaxLinks);
      return bad(buf);
    }
    int nq = 0, nv = 0, ncs = 0, nlim = 0;
    for (int l = 0; l < n; ++l) {
      const int i = o0 + l;
      if (d->limits) {
        const double lo = d->limits[2 * i], hi = d->limits[2 * i + 1];
        if (std::isnan(lo) || std::isnan(hi) || !(lo < hi) || lo == INFINITY || hi == -INFINITY) {
          snprintf(buf, sizeof buf, "system %d link %d: joint limits need lo < hi", b, l);
          return bad(buf);
        }
        if (std::isfinite(lo) || std::isfinite(hi)) {
          if (d->joint_type[i] != SIM_REVOLUTE) {
            snprintf(buf, sizeof buf, "system %d link %d: limits apply to revolute joints only", b, l);
            return bad(buf);
          }
          ++nlim;
        }
      }
      if (d->contact) {
        const double* c = d->contact + 4 * i;
        for (int x = 0; x < 4; ++x)
          if (!std::isfinite(c[x])) return bad("non-finite contact sphere");
        if (c[3] >= 0) ++ncs;
      }
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
    if (ncs > SIM_MAX_CONTACTS) {
      snprintf(buf, sizeof buf, "system %d has %d contact spheres (at most %d)", b, ncs, SIM_MAX_CONTACTS);
      return bad(buf);
    }
    if (nlim > SIM_MAX_LIMITS) {
      snprintf(buf, sizeof buf, "system %d has %d limited joints (at most %d)", b, nlim, SIM_MAX_LIMITS);
      return bad(buf);
    }
    any_contact |= ncs > 0 || nlim > 0;
  }
  if (any_contact) {
    if (!(d->friction >= 0) || !std::isfinite(d->friction)) return bad("friction must be finite and >= 0");
    if (!(d->erp >= 0 && d->erp <= 1)) return bad("erp must be in [0, 1]");
    if (d->pgs_iterations < 1 || d->pgs_iterations > SIM_MAX_PGS_ITERATIONS)
      return bad("pgs_iterations must be in [1, SIM_MAX_PGS_ITERATIONS]");
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

// ------------------------------------------------------------------ static scratch
// Per-link tape for sim_step_batch_static: a file-scope device array, so that
// entry point needs no allocation at all.  Every GPU that loads this library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_tape[SIM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_tape on the handle's device, which must be current,
// looked up once per device (the symbol's name in host code is only a host-side
// stand-in, never a device address).
int static_tape(sim_handle* h, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "static scratch: cudaGetDevice");
  if (dev != h->device)
    return fail(h, SIM_EINVAL, "static scratch: make the handle's device (current at sim_create) current");
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
  return launch_step_with_tape<T, DT>(h, q, qd, tau, q_out, qd_out, tape, stream);
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
  if (!(d->flags & SIM_KEEP_SYSTEM_ORDER))
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nl_sys[x] > nl_sys[y]; });
  h->h_sys_of_slot = order;
  const int maxL = h->maxL;
  const size_t Bpad = (size_t)((B + LANES - 1) / LANES) * LANES;
  h->Bpad = (int)Bpad;
  std::vector<int> nl(B), nqv(B);
  std::vector<double> prm((size_t)maxL * NPRM * Bpad, 0.0);
  std::vector<int> meta((size_t)maxL * Bpad, 0), slot(h->L_total);
  // per link: the frame change R (x' = R x) that puts a revolute axis on z.  With
  // R_p the parent's (identity for the world): X_tree' = (R E_t R_p^T, R_p r_t),
  // com' = R com, I_com' = R I_com R^T, sphere centre' = R p.  States, inputs and
  // every gradient are in joint coordinates, so none of them changes.
  const M9 eye{1, 0, 0, 0, 1, 0, 0, 0, 1};
  std::vector<M9> Rl(h->L_total, eye);
  for (int i = 0; i < h->L_total; ++i)
    if (d->joint_type[i] == SIM_REVOLUTE) Rl[i] = rotation_to_z(d->axis + 3 * i);
  bool any_contact = false;
  for (int sl = 0; sl < B; ++sl) {
    const int b = order[sl];
    nl[sl] = nl_sys[b];
    const int n = nl[sl], o = d->sys_link_offset[b];
    // coordinates keep the model's numbering; the links are stored in depth-first
    // preorder (perm: stored position -> model link), children in model order
    std::vector<int> qoff(n), voff(n);
    int qo = 0, vo = 0;
    for (int l = 0; l < n; ++l) {
      qoff[l] = qo;
      voff[l] = vo;
      qo += d->joint_type[o + l] == SIM_FREE ? 7 : 1;
      vo += d->joint_type[o + l] == SIM_FREE ? 6 : 1;
    }
    const TreeOrder to = tree_order(d->parent + o, n);
    const std::vector<int>& perm = to.perm;
    h->wdepth = std::max(h->wdepth, to.depth);
    for (int l = 0; l < n; ++l) {
      const int i = o + perm[l];
      const int jt = d->joint_type[i];
      const size_t tile = sl / LANES, lane = sl % LANES;
      auto P = [&](int f) -> double& { return prm[((tile * maxL + l) * NPRM + f) * LANES + lane]; };
      const M9& R = Rl[i];
      const M9& Rp = d->parent[i] >= 0 ? Rl[d->sys_link_offset[b] + d->parent[i]] : eye;
      M9 Et;
      for (int x = 0; x < 9; ++x) Et[x] = d->X_tree[12 * i + x];
      const M9 Et2 = mat_mul(mat_mul(R, Et), mat_T(Rp));
      double rt[3], com[3], cp[3] = {0, 0, 0};
      mat_vec(Rp, d->X_tree + 12 * i + 9, rt);
      mat_vec(R, d->com + 3 * i, com);
      if (d->contact) mat_vec(R, d->contact + 4 * i, cp);
      const double* ic = d->I_com + 6 * i;  // xx yy zz xy xz yz
      const M9 Ic2 = mat_mul(mat_mul(R, M9{ic[0], ic[3], ic[4], ic[3], ic[1], ic[5], ic[4], ic[5], ic[2]}), mat_T(R));
      for (int x = 0; x < 9; ++x) P(P_E + x) = Et2[x];
      for (int x = 0; x < 3; ++x) {
        P(P_R + x) = rt[x];
        P(P_AX + x) = (jt == SIM_REVOLUTE && x == 2) ? 1.0 : 0.0;
        P(P_C + x) = com[x];
        P(P_CP + x) = cp[x];
      }
      P(P_M) = d->mass[i];
      const double ic2[6] = {Ic2[0], Ic2[4], Ic2[8], Ic2[1], Ic2[2], Ic2[5]};
      for (int x = 0; x < 6; ++x) P(P_IC + x) = ic2[x];
      P(P_DAMP) = (d->damping && jt == SIM_REVOLUTE) ? d->damping[i] : 0.0;
      P(P_CR) = (d->contact && d->contact[4 * i + 3] >= 0) ? d->contact[4 * i + 3] : -1.0;
      if (d->contact && d->contact[4 * i + 3] >= 0) any_contact = true;
      const bool lim = d->limits && jt == SIM_REVOLUTE;
      P(P_LO) = lim ? d->limits[2 * i] : -INFINITY;
      P(P_HI) = lim ? d->limits[2 * i + 1] : INFINITY;
      if (lim && (std::isfinite(d->limits[2 * i]) || std::isfinite(d->limits[2 * i + 1]))) any_contact = true;
      meta[(tile * maxL + l) * LANES + lane] =
          make_meta(to.parent[l], jt, to.branch[l], qoff[perm[l]], voff[perm[l]], to.lastsib[l]);
      slot[i] = l * B + sl;
    }
    nqv[sl] = qo | (vo << 16);
    h->nq_max = std::max(h->nq_max, qo);
    h->nv_max = std::max(h->nv_max, vo);
  }
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  h->all_chains = !any_contact;
  h->all_revolute = !any_contact;
  for (int i = 0; i < h->L_total && h->all_revolute; ++i)
    if (d->joint_type[i] != SIM_REVOLUTE) h->all_revolute = false;
  for (int b = 0; b < B && h->all_chains; ++b)
    for (int l = 0; l < nl_sys[b]; ++l) {
      const int i = d->sys_link_offset[b] + l;
      if (d->joint_type[i] != SIM_REVOLUTE || d->parent[i] != l - 1) h->all_chains = false;
    }
  // the pipelined kernels take a tile's first slot as its longest system
  for (int b = 1; b < B && h->all_chains; ++b)
    if (nl_sys[order[b]] > nl_sys[order[(b / LANES) * LANES]]) h->all_chains = false;
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
  if (rc == SIM_OK && h->all_revolute)
    rc = alloc(&h->wtape2, (size_t)maxL * NWT * Bpad * h->scalar, "second world-aligned tape");
  if (rc == SIM_OK && h->all_revolute && h->wdepth > 0)
    rc = alloc(&h->wstk, (size_t)2 * h->wdepth * WSW * Bpad * h->scalar, "world-aligned stacks");
  if (rc == SIM_OK) rc = alloc((void**)&h->status, B * sizeof(int), "status");
  if (rc == SIM_OK) rc = alloc((void**)&h->sys_of_slot, B * sizeof(int), "slot order");
  if (rc == SIM_OK) rc = put(h->sys_of_slot, order.data(), B * sizeof(int));
  if (rc == SIM_OK) rc = alloc((void**)&h->counter, sizeof(unsigned), "work ticket");
  if (any_contact) {
    h->friction = d->friction;
    h->erp = d->erp;
    h->pgs_iterations = d->pgs_iterations;
    if (rc == SIM_OK) rc = alloc(&h->ctape, (size_t)maxL * NCT * Bpad * h->scalar, "contact tape");
    if (rc == SIM_OK) rc = alloc(&h->csys, (size_t)NCS * Bpad * h->scalar, "contact record");
  }
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
                  h->status, h->sys_of_slot, h->counter, h->ctape, h->csys, h->x64, h->wtape2, h->wstk};
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
  return is_fp64(h) ? launch_set_masses<double>(h, mass, stream) : launch_set_masses<float>(h, mass, stream);
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
  if (h->ctape) return fail(h, SIM_EUNSUPPORTED, "forward-mode step of a model with contact spheres or limits");
  return is_fp64(h) ? launch_jvp<double>(h, q, qd, tau, dq, dqd, dtau, q_out, qd_out, dq_out, dqd_out, work, stream)
                    : launch_jvp<float>(h, q, qd, tau, dq, dqd, dtau, q_out, qd_out, dq_out, dqd_out, work, stream);
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
  if (space != SIM_TAPE_AUTO && space != SIM_TAPE_GLOBAL && space != SIM_TAPE_SHARED &&
      space != SIM_TAPE_PIPELINED && space != SIM_TAPE_ONE_WARP && space != SIM_TAPE_ALIGNED &&
      space != SIM_TAPE_ALIGNED_PIPELINED)
    return fail(h, SIM_EINVAL, "unknown tape space");
  h->tape_space = space;
  return SIM_OK;
}

int sim_last_storage(const sim_handle* h, int32_t* rollout_mode, int32_t* backward_mode) {
  if (!h) return SIM_EINVAL;
  if (rollout_mode) *rollout_mode = h->last_storage;
  if (backward_mode) *backward_mode = h->last_storage_bwd;
  return SIM_OK;
}

int sim_set_prefetch(sim_handle* h, int32_t links_ahead) {
  if (!h) return SIM_EINVAL;
  if (links_ahead < 0 || links_ahead > 16) return fail(h, SIM_EINVAL, "prefetch distance must be in [0, 16]");
  h->prefetch = links_ahead;
  return SIM_OK;
}

int sim_set_replay(sim_handle* h, int32_t mode) {
  if (!h) return SIM_EINVAL;
  if (mode != SIM_REPLAY_SEGMENT && mode != SIM_REPLAY_QUADRATIC) return fail(h, SIM_EINVAL, "unknown replay mode");
  h->replay = mode;
  return SIM_OK;
}

int sim_set_state_accumulation(sim_handle* h, int32_t fp64) {
  if (!h) return SIM_EINVAL;
  if (fp64 != 0 && fp64 != 1) return fail(h, SIM_EINVAL, "state accumulation flag must be 0 or 1");
  if (fp64 && h->precision != SIM_FP32_D64)
    return fail(h, SIM_EUNSUPPORTED, "FP64 state accumulation applies to the FP32 + FP64 D-solve mode");
  if (fp64 && !h->x64) {
    cudaError_t e = cudaMalloc(&h->x64, (size_t)(h->nq_max + h->nv_max) * h->B * sizeof(double));
    if (e != cudaSuccess) {
      h->x64 = nullptr;
      return cuda_fail(h, e, "FP64 state buffer");
    }
  }
  h->state64 = fp64 != 0;
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
