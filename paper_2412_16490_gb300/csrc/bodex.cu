// BODex coarse-stage hot path for GB300 (sm_103a): the C ABI declared in
// include/bodex.h and its small kernels (kinematics, refinement, metrics);
// the heavy kernels live in bodex_kernels.cuh and are compiled in their own
// translation units.
//
// Kernel layout.  One CTA holds GPB grasps and s lanes (threads) per grasp,
// GPB * s = 96 threads for s = 6 or 12.  Lane j of a grasp owns the QP of
// desired wrench t_j and keeps its ADMM iterate (y: 3m, w: 9m+1 floats) in
// registers; the grasp's G and explicit K^-1 sit in shared memory and are
// read by all of its lanes.  Lanes 0..m-1 also own one contact each for the
// kinematics, the SDF query and the adjoint.  The fused step kernel runs
// every upper iteration of a launch back to back without leaving the CTA:
// pose, Adam moments and warm starts never return to HBM between steps.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bodex.h"
#include "bodex_device.cuh"
#include "bodex_kernels.cuh"

using namespace bodex;

// ============================================================================ error state
namespace {
thread_local std::string g_err;
}  // namespace

namespace bodex {
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  return fail(BODEX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
int launch_err(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return BODEX_OK;
}
}  // namespace bodex

#define BODEX_CUDA(call)                                    \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

namespace {
cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
}  // namespace

struct bodex_hand_s {
  HandDev host;
  HandDev* dev = nullptr;
  float* tips = nullptr;  // [m, S, 3] fingertip surface samples (refinement)
  void* coll_mem = nullptr;  // collision spheres (one allocation behind coll's pointers)
  CollDev coll{};
};
struct bodex_object_s {
  ObjDev dev;
  float* grid = nullptr;
};
struct bodex_state_s {
  int B = 0, s = 0, m = 0, D = 0;
  float* x = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  // ADMM warm start, component-major ([3m][B s] and [9m+1][B s]) so that the
  // fused kernel's per-step loads and stores are coalesced across lanes
  float* qy = nullptr;
  float* qw = nullptr;
  float* res = nullptr;  // [B] max QP residual at the last step of the last launch
  int* work = nullptr;   // work-item counter of a several-job launch led by this state
  int t = 0;
};

// ============================================================================ kernel: FK + contacts + G
template <int M>
__global__ void __launch_bounds__(128) fk_contacts_kernel(const HandDev* __restrict__ hand, ObjDev obj,
                                                          const float* __restrict__ x, int B, float* c_w,
                                                          float* p_out, float* n_out, float* phi_out, float* G_out,
                                                          int32_t* cell_out, int32_t* status_out) {
  __shared__ __align__(16) float hs[Lay<M>::HAND_WORDS];
  copy_hand_to_smem(hand, hs);
  __syncthreads();
  const HandDev& H = *reinterpret_cast<const HandDev*>(hs);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  constexpr int NV = 3 * M;
  const int D = H.D;
  float xl[MAXD];
  int st = 0;
  for (int k = 0; k < D; ++k) {
    xl[k] = x[(size_t)b * D + k];
    if (!isfinite(xl[k])) st |= BODEX_ST_NONFINITE;
  }
  float Gl[6 * NV];
  for (int i = 0; i < M; ++i) {
    float c[3];
    fk_contact(H, i, xl, c, nullptr);
    const ContactGeo k = contact_geometry(obj, c);
    if (k.degenerate) st |= BODEX_ST_DEGENERATE_NORMAL;
    if (!finite3(k.p) || !finite3(k.n) || !isfinite(k.phi)) st |= BODEX_ST_NONFINITE;
    write_G_block(k, i, NV, Gl);
    const size_t o = ((size_t)b * M + i) * 3;
    const float gc[3] = {obj.gcx, obj.gcy, obj.gcz};
    for (int a = 0; a < 3; ++a) {
      if (c_w) c_w[o + a] = k.c[a];
      if (p_out) p_out[o + a] = k.p[a] + gc[a];
      if (n_out) n_out[o + a] = k.n[a];
      if (cell_out) cell_out[o + a] = k.cell[a];
    }
    if (phi_out) phi_out[(size_t)b * M + i] = k.phi;
  }
  if (G_out)
    for (int e = 0; e < 6 * NV; ++e) G_out[(size_t)b * 6 * NV + e] = Gl[e];
  if (status_out) status_out[b] = st;
}

// ============================================================================ kernel: refinement epilogue
// Fine / final stages (Sec. IV-C, Eqs. (10)-(11)) in SDF form, no QP.  Per
// contact: c^f = the fingertip sample with the smallest phi (lowest index on
// ties), p^f its nearest object point, c^{f'} = R_i s_{k*} + T_i with the
// sample's link-frame coordinates held fixed (the Detach of Eq. (11)), and
//   E = w_d sum |c^{f'} - (p^f + delta n_out)|^2 + w_qp sum |c^{f'} - p^c|^2
// with p^f, n_out and the coarse-stage points p^c treated as constants.
// delta is the pre-grasp margin (Sec. IV-D): 1 cm in the fine stage, 0 in
// the final one.  One CTA holds RF_GPB grasps x 8 lanes; lanes 0..m-1 own a
// contact, all lanes share the gradient assembly and Adam.
struct RefineArgs {
  const HandDev* hand;
  const float* tips;
  ObjDev obj;
  int B;
  const float* pc;
  float delta, w_d, w_qp;
  float lr_t, lr_r, b1, b2, adam_eps;
  int n_steps, t0;
  float* x;
  float* am;
  float* av;
  float* E;
  int32_t* kstar;
  int32_t* status;
};

constexpr int RF_LANES = 8, RF_GPB = 16;

template <int M>
__global__ void __launch_bounds__(RF_LANES * RF_GPB) refine_kernel(RefineArgs A) {
  constexpr int HW = Lay<M>::HAND_WORDS;
  constexpr int CBW = 6 + MAXCHAIN;
  constexpr int PER = align4(3 * MAXD + M * CBW + M * MAXCHAIN * 6 + M + 4);
  __shared__ __align__(16) float smem[HW + RF_GPB * PER];
  copy_hand_to_smem(A.hand, smem);
  const int gl = threadIdx.x / RF_LANES, lane = threadIdx.x % RF_LANES;
  const int b = blockIdx.x * RF_GPB + gl;
  const bool active = b < A.B;
  const HandDev& H = *reinterpret_cast<const HandDev*>(smem);
  float* per = smem + HW + gl * PER;
  float* xs = per;
  float* ams = per + MAXD;
  float* avs = per + 2 * MAXD;
  float* cb = per + 3 * MAXD;
  float* jwall = cb + M * CBW;
  float* Ei = jwall + M * MAXCHAIN * 6;
  int* stat = reinterpret_cast<int*>(Ei + M);
  __syncthreads();
  const int D = H.D, S = H.S;
  if (active) {
    for (int k = lane; k < D; k += RF_LANES) {
      xs[k] = A.x[(size_t)b * D + k];
      ams[k] = A.am[(size_t)b * D + k];
      avs[k] = A.av[(size_t)b * D + k];
    }
    if (lane == 0) *stat = 0;
  }
  __syncthreads();
  int kbest = 0;
  for (int step = 0; step < A.n_steps; ++step) {
    if (active && lane < M) {
      Tf T;
      float* jw = jwall + lane * MAXCHAIN * 6;
      fk_link(H, lane, xs, T, jw);
      const float* tip = A.tips + (size_t)lane * S * 3;
      float best = INFINITY;
      kbest = 0;
      for (int k = 0; k < S; ++k) {
        const float sk[3] = {__ldg(tip + 3 * k), __ldg(tip + 3 * k + 1), __ldg(tip + 3 * k + 2)};
        float ck[3];
        tf_point(T, sk, ck);
        const float ph = sdf_query(A.obj, ck).phi;
        if (ph < best) {
          best = ph;
          kbest = k;
        }
      }
      const float sk[3] = {__ldg(tip + 3 * kbest), __ldg(tip + 3 * kbest + 1), __ldg(tip + 3 * kbest + 2)};
      float cf[3];
      tf_point(T, sk, cf);
      const ContactGeo k = contact_geometry(A.obj, cf);
      const float gc[3] = {A.obj.gcx, A.obj.gcy, A.obj.gcz};
      const float* pci = A.pc + ((size_t)b * M + lane) * 3;
      float dEdc[3], e = 0.f;
      for (int a = 0; a < 3; ++a) {
        const float target = k.p[a] + gc[a] - A.delta * k.n[a];
        const float da = cf[a] - target, db = cf[a] - pci[a];
        e += A.w_d * da * da + A.w_qp * db * db;
        dEdc[a] = 2.f * A.w_d * da + 2.f * A.w_qp * db;
      }
      Ei[lane] = e;
      if (k.degenerate) atomicOr(stat, BODEX_ST_DEGENERATE_NORMAL);
      if (!isfinite(e)) atomicOr(stat, BODEX_ST_NONFINITE);
      float* c = cb + lane * CBW;
      c[0] = dEdc[0];
      c[1] = dEdc[1];
      c[2] = dEdc[2];
      float s1, c1, s2, c2;
      angle_sincos(xs[3], &s1, &c1);
      angle_sincos(xs[4], &s2, &c2);
      const float om[3][3] = {{1.f, 0.f, 0.f}, {0.f, c1, s1}, {s2, -s1 * c2, c1 * c2}};
      const float rel[3] = {cf[0] - xs[0], cf[1] - xs[1], cf[2] - xs[2]};
      for (int k3 = 0; k3 < 3; ++k3) {
        float v[3];
        cross3(om[k3], rel, v);
        c[3 + k3] = dEdc[0] * v[0] + dEdc[1] * v[1] + dEdc[2] * v[2];
      }
      const int Lc = H.chain_len[lane];
      for (int kk = 0; kk < Lc; ++kk) {
        const float r2[3] = {cf[0] - jw[6 * kk + 3], cf[1] - jw[6 * kk + 4], cf[2] - jw[6 * kk + 5]};
        float v[3];
        cross3(jw + 6 * kk, r2, v);
        c[6 + kk] = dEdc[0] * v[0] + dEdc[1] * v[1] + dEdc[2] * v[2];
      }
    }
    __syncthreads();
    if (active) {
      const int tstep = A.t0 + step + 1;
      const float c1 = 1.f - exp2f((float)tstep * log2f(A.b1)), c2 = 1.f - exp2f((float)tstep * log2f(A.b2));
      if (lane == 0 && A.E) {
        float e = 0.f;
        for (int i = 0; i < M; ++i) e += Ei[i];
        per[PER - 1] = e;
      }
      for (int k = lane; k < D; k += RF_LANES) {
        float g = 0.f;
        if (k < 6) {
          for (int i = 0; i < M; ++i) g += cb[i * CBW + k];
        } else {
          for (int i = 0; i < M; ++i) {
            const int pos = H.jpos[i][k - 6];
            if (pos >= 0) g += cb[i * CBW + 6 + pos];
          }
        }
        const float mm = fmaf(A.b1, ams[k], (1.f - A.b1) * g);
        const float vv = fmaf(A.b2, avs[k], (1.f - A.b2) * g * g);
        ams[k] = mm;
        avs[k] = vv;
        const float lr = k < 3 ? A.lr_t : A.lr_r;
        const float xn = xs[k] - lr * (mm / c1) / (sqrtf(vv / c2) + A.adam_eps);
        xs[k] = fminf(fmaxf(xn, H.qmin[k]), H.qmax[k]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  for (int k = lane; k < D; k += RF_LANES) {
    A.x[(size_t)b * D + k] = xs[k];
    A.am[(size_t)b * D + k] = ams[k];
    A.av[(size_t)b * D + k] = avs[k];
  }
  if (lane < M && A.kstar && A.n_steps > 0) A.kstar[(size_t)b * M + lane] = kbest;
  if (lane == 0) {
    if (A.E) A.E[b] = per[PER - 1];
    if (A.status) A.status[b] = *stat;
  }
}

// ============================================================================ kernel: contact metrics
// Contact Distance Consistency (Sec. V-B): d_i = the signed distance of
// fingertip i, the smallest phi over its surface samples (phi(c_i) - alpha
// for a hand without samples); cdc = max_i d_i - min_i d_i.  Eight lanes per
// grasp, lane i < m owns finger i; the spread is reduced across the lanes.
struct MetricsArgs {
  const HandDev* hand;
  const float* tips;  // [m, S, 3] or null
  ObjDev obj;
  int B;
  const float* x;
  float* d;    // [B, m]
  float* cdc;  // [B], may be null
};

template <int M>
__global__ void __launch_bounds__(RF_LANES * RF_GPB) metrics_kernel(MetricsArgs A) {
  constexpr int HW = Lay<M>::HAND_WORDS;
  constexpr int XW = align4(MAXD);
  __shared__ __align__(16) float smem[HW + RF_GPB * XW];
  copy_hand_to_smem(A.hand, smem);
  const int gl = threadIdx.x / RF_LANES, lane = threadIdx.x % RF_LANES;
  const int b = blockIdx.x * RF_GPB + gl;
  const bool active = b < A.B;
  const HandDev& H = *reinterpret_cast<const HandDev*>(smem);
  float* xs = smem + HW + gl * XW;
  __syncthreads();
  const int D = H.D, S = A.tips ? H.S : 0;
  if (active)
    for (int k = lane; k < D; k += RF_LANES) xs[k] = A.x[(size_t)b * D + k];
  __syncthreads();
  const bool mine = active && lane < M;
  float d = 0.f;
  if (mine) {
    Tf T;
    fk_link(H, lane, xs, T, nullptr);
    if (S > 0) {
      const float* tip = A.tips + (size_t)lane * S * 3;
      d = INFINITY;
      for (int k = 0; k < S; ++k) {
        const float sk[3] = {__ldg(tip + 3 * k), __ldg(tip + 3 * k + 1), __ldg(tip + 3 * k + 2)};
        float ck[3];
        tf_point(T, sk, ck);
        d = fminf(d, sdf_query(A.obj, ck).phi);
      }
    } else {
      float c[3];
      tf_point(T, H.clocal[lane], c);
      d = sdf_query(A.obj, c).phi - H.alpha;
    }
    A.d[(size_t)b * M + lane] = d;
  }
  // spread over the grasp's fingers (all lanes of the 8-lane group take part)
  float lo = mine ? d : INFINITY, hi = mine ? d : -INFINITY;
#pragma unroll
  for (int off = RF_LANES / 2; off >= 1; off >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off, RF_LANES));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off, RF_LANES));
  }
  if (active && lane == 0 && A.cdc) A.cdc[b] = hi - lo;
}

// ============================================================================ host helpers
namespace {

int check_qp_params(const bodex_qp_params* p, int m) {
  if (!p) return fail(BODEX_ERR_INVALID, "null qp params");
  if (!(p->gamma >= 0.f) || p->gamma > (float)m)
    return fail(BODEX_ERR_INFEASIBLE, "gamma must lie in [0, m]");
  if (!(p->rho > 0.f) || !(p->sigma >= 0.f) || !(p->alpha > 0.f && p->alpha < 2.f) || p->max_iter < 0 ||
      !(p->mu >= 0.f))
    return fail(BODEX_ERR_INVALID, "invalid ADMM parameters");
  if (p->cone != BODEX_CONE_PYRAMID && p->cone != BODEX_CONE_ELLIPTIC)
    return fail(BODEX_ERR_INVALID, "cone must be BODEX_CONE_PYRAMID or BODEX_CONE_ELLIPTIC");
  if (p->solver != BODEX_QP_ADMM && p->solver != BODEX_QP_EXACT)
    return fail(BODEX_ERR_INVALID, "solver must be BODEX_QP_ADMM or BODEX_QP_EXACT");
  if (p->polish < 0 || p->polish > 2) return fail(BODEX_ERR_INVALID, "polish must be 0, 1 or 2");
  if (p->solver == BODEX_QP_EXACT && (p->cone != BODEX_CONE_PYRAMID || p->eps_reg != 0.f || p->max_iter < 1))
    return fail(BODEX_ERR_INVALID, "the exact solver needs the pyramid cone, eps_reg = 0 and max_iter >= 1");
  return BODEX_OK;
}

int dispatch_fused(int m, int mode, const FusedArgs& A, cudaStream_t st) {
  switch (m) {
    case 3: return launch_fused_m3(mode, A, st);
    case 4: return launch_fused_m4(mode, A, st);
    case 5: return launch_fused_m5(mode, A, st);
    default: return fail(BODEX_ERR_INVALID, "m must be 3, 4 or 5");
  }
}

template <int M>
int run_fk(const bodex_hand_s* h, const bodex_object_s* o, const float* x, int B, float* c_w, float* p, float* n,
           float* phi, float* G, int32_t* cell, int32_t* status, cudaStream_t st) {
  if (B == 0) return BODEX_OK;
  (void)cudaGetLastError();
  fk_contacts_kernel<M><<<(B + 127) / 128, 128, 0, st>>>(h->dev, o->dev, x, B, c_w, p, n, phi, G, cell, status);
  return launch_err("fk_contacts_kernel launch");
}

}  // namespace

namespace {
template <int M>
int run_refine(const RefineArgs& A, cudaStream_t st) {
  (void)cudaGetLastError();
  refine_kernel<M><<<(A.B + RF_GPB - 1) / RF_GPB, RF_LANES * RF_GPB, 0, st>>>(A);
  return launch_err("refine_kernel launch");
}

template <int M>
int run_metrics(const MetricsArgs& A, cudaStream_t st) {
  (void)cudaGetLastError();
  metrics_kernel<M><<<(A.B + RF_GPB - 1) / RF_GPB, RF_LANES * RF_GPB, 0, st>>>(A);
  return launch_err("metrics_kernel launch");
}
}  // namespace

// ============================================================================ hand collision spheres
// Shared-memory room the fused kernel has for the collision scratch of one
// grasp (sphere centres and per-slot sums), by contact count.
static int coll_room(int m) {
  switch (m) {
    case 3: return Lay<3>::COLL_CS;
    case 4: return Lay<4>::COLL_CS;
    default: return Lay<5>::COLL_CS;
  }
}
static int frame_room(int m) {
  switch (m) {
    case 3: return Lay<3>::COLL_FR;
    case 4: return Lay<4>::COLL_FR;
    default: return Lay<5>::COLL_FR;
  }
}

// Orders the spheres by slot (link, then the root), bounds each slot's
// spheres, lists the slot pairs allowed for self-penetration, and uploads
// them in one allocation.  Pair rule: spheres on different links, except a
// link and its nearest ancestor link that carries spheres (the root counts).
static int upload_spheres(bodex_hand_s* h, const bodex_hand_desc* d) {
  const int K = d->n_spheres, n = h->host.n;
  if (K == 0) return BODEX_OK;
  if (K < 0 || K > BODEX_MAX_SPHERES) return fail(BODEX_ERR_INVALID, "n_spheres out of range");
  if (!d->sphere_link || !d->sphere_local || !d->sphere_radius)
    return fail(BODEX_ERR_INVALID, "null sphere array in hand descriptor");
  std::vector<int> slot(K);
  for (int k = 0; k < K; ++k) {
    const int L = d->sphere_link[k];
    if (L < -1 || L >= n) return fail(BODEX_ERR_INVALID, "sphere_link out of range");
    if (!(d->sphere_radius[k] > 0.f)) return fail(BODEX_ERR_INVALID, "sphere_radius must be > 0");
    slot[k] = L < 0 ? n : L;
  }

  if (3 * K + 9 * (n + 1) > coll_room(h->host.m) || 12 * (n + 1) > frame_room(h->host.m))
    return fail(BODEX_ERR_INVALID, "too many collision spheres and joints for this contact count");
  // the collision phase takes its link frames from the contact kinematics
  for (int k = 0; k < K; ++k) {
    const int L = d->sphere_link[k];
    bool on_chain = L < 0;
    for (int i = 0; i < h->host.m && !on_chain; ++i) on_chain = h->host.jpos[i][L] >= 0;
    if (!on_chain) return fail(BODEX_ERR_INVALID, "a sphere link lies on no contact chain");
  }
  std::vector<int> order(K);
  for (int k = 0; k < K; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return slot[a] < slot[b]; });
  std::vector<char> has(n, 0);
  for (int k = 0; k < K; ++k)
    if (d->sphere_link[k] >= 0) has[d->sphere_link[k]] = 1;
  auto eff_parent = [&](int L) {  // -1: the root; -2: none (L is the root)
    if (L < 0) return -2;
    int p = h->host.parent[L];
    while (p >= 0 && !has[p]) p = h->host.parent[p];
    return p;
  };
  std::vector<float4> sph(K);
  std::vector<int> slot_start(n + 2, 0);
  for (int a = 0; a < K; ++a) {
    const int ka = order[a];
    sph[a] = make_float4(d->sphere_local[3 * ka], d->sphere_local[3 * ka + 1], d->sphere_local[3 * ka + 2],
                         d->sphere_radius[ka]);
    ++slot_start[slot[ka] + 1];
  }
  for (int L = 0; L <= n; ++L) slot_start[L + 1] += slot_start[L];
  // bounding sphere of each slot's spheres (centre: their mean), and the
  // slot pairs allowed for self-penetration
  std::vector<float4> sbound(n + 1, make_float4(0.f, 0.f, 0.f, 0.f));
  for (int L = 0; L <= n; ++L) {
    const int k0 = slot_start[L], k1 = slot_start[L + 1];
    if (k0 == k1) continue;
    double c[3] = {0, 0, 0};
    for (int k = k0; k < k1; ++k) {
      c[0] += sph[k].x;
      c[1] += sph[k].y;
      c[2] += sph[k].z;
    }
    for (double& v : c) v /= (k1 - k0);
    double R = 0;
    for (int k = k0; k < k1; ++k) {
      const double dx = sph[k].x - c[0], dy = sph[k].y - c[1], dz = sph[k].z - c[2];
      R = std::max(R, std::sqrt(dx * dx + dy * dy + dz * dz) + sph[k].w);
    }
    sbound[L] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)(R * (1.0 + 1e-5)) + 1e-6f);
  }
  auto link_of = [&](int L) { return L == n ? -1 : L; };
  std::vector<int> spstart(n + 2, 0), spartners;
  for (int L = 0; L <= n; ++L) {
    for (int L2 = 0; L2 <= n; ++L2) {
      if (L2 == L || slot_start[L] == slot_start[L + 1] || slot_start[L2] == slot_start[L2 + 1]) continue;
      const int la = link_of(L), lb = link_of(L2);
      if (eff_parent(la) == lb || eff_parent(lb) == la) continue;
      spartners.push_back(L2);
    }
    spstart[L + 1] = (int)spartners.size();
  }
  const size_t b_sph = sizeof(float4) * K, b_sb = sizeof(float4) * (n + 1), b_ss = sizeof(int) * (n + 2),
               b_sp = sizeof(int) * (n + 2), b_pa = sizeof(int) * std::max<size_t>(1, spartners.size());
  const size_t o_sb = b_sph, o_ss = o_sb + b_sb, o_sp = o_ss + b_ss, o_pa = o_sp + b_sp;
  std::vector<char> blob(o_pa + b_pa);
  std::memcpy(blob.data(), sph.data(), b_sph);
  std::memcpy(blob.data() + o_sb, sbound.data(), b_sb);
  std::memcpy(blob.data() + o_ss, slot_start.data(), b_ss);
  std::memcpy(blob.data() + o_sp, spstart.data(), b_sp);
  if (!spartners.empty()) std::memcpy(blob.data() + o_pa, spartners.data(), sizeof(int) * spartners.size());
  if (cudaMalloc(&h->coll_mem, blob.size()) != cudaSuccess) {
    h->coll_mem = nullptr;
    return fail(BODEX_ERR_OOM, "cudaMalloc collision spheres");
  }
  cudaError_t e = cudaMemcpy(h->coll_mem, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy collision spheres");
  char* base = static_cast<char*>(h->coll_mem);
  h->coll.K = K;
  h->coll.sph = reinterpret_cast<const float4*>(base);
  h->coll.sbound = reinterpret_cast<const float4*>(base + o_sb);
  h->coll.slot_start = reinterpret_cast<const int*>(base + o_ss);
  h->coll.spstart = reinterpret_cast<const int*>(base + o_sp);
  h->coll.spartners = reinterpret_cast<const int*>(base + o_pa);
  return BODEX_OK;
}

extern "C" int bodex_hand_destroy(bodex_hand_t h);

// ============================================================================ C ABI
extern "C" {

const char* bodex_last_error(void) { return g_err.c_str(); }
const char* bodex_version(void) { return "bodex-gb300 0.1 (sm_103a)"; }

int bodex_step_tile(int m, int s, int requested, int* grasps_per_cta) {
  if (!grasps_per_cta || s < 1 || s > SMAX || requested < 0)
    return fail(BODEX_ERR_INVALID, "bodex_step_tile: s outside 1..16, requested < 0 or null output");
  switch (m) {
    case 3: *grasps_per_cta = pick_gpb<3>(s, requested); break;
    case 4: *grasps_per_cta = pick_gpb<4>(s, requested); break;
    case 5: *grasps_per_cta = pick_gpb<5>(s, requested); break;
    default: return fail(BODEX_ERR_INVALID, "bodex_step_tile: m must be 3, 4 or 5");
  }
  return BODEX_OK;
}

int bodex_sync(void* stream) {
  BODEX_CUDA(cudaStreamSynchronize(as_stream(stream)));
  return BODEX_OK;
}

int bodex_hand_create(const bodex_hand_desc* d, bodex_hand_t* out) {
  if (!d || !out) return fail(BODEX_ERR_INVALID, "null argument");
  *out = nullptr;
  const int n = d->n_joints, m = d->n_contacts;
  if (n < 1 || n > MAXJ) return fail(BODEX_ERR_INVALID, "n_joints out of range");
  if (m < 3 || m > MAXM) return fail(BODEX_ERR_INVALID, "n_contacts must be 3..5");
  if (!d->parent || !d->offset || !d->axis || !d->qmin || !d->qmax || !d->contact_link || !d->contact_local)
    return fail(BODEX_ERR_INVALID, "null array in hand descriptor");
  HandDev H;
  std::memset(&H, 0, sizeof(H));
  H.n = n;
  H.m = m;
  H.D = 6 + n;
  H.alpha = d->contact_radius;
  H.S = d->n_tip_samples;
  for (int j = 0; j < n; ++j) {
    H.parent[j] = d->parent[j];
    if (H.parent[j] >= j || H.parent[j] < -1) return fail(BODEX_ERR_INVALID, "parent[j] must be -1 or < j");
    for (int e = 0; e < 12; ++e) H.offset[j][e] = d->offset[12 * j + e];
    for (int e = 0; e < 3; ++e) H.axis[j][e] = d->axis[3 * j + e];
  }
  for (int k = 0; k < 6 + n; ++k) {
    H.qmin[k] = d->qmin[k];
    H.qmax[k] = d->qmax[k];
    if (!(H.qmin[k] <= H.qmax[k])) return fail(BODEX_ERR_INFEASIBLE, "qmin > qmax");
  }
  for (int i = 0; i < MAXM; ++i)
    for (int j = 0; j < MAXJ; ++j) H.jpos[i][j] = -1;
  for (int i = 0; i < m; ++i) {
    H.clink[i] = d->contact_link[i];
    if (H.clink[i] < 0 || H.clink[i] >= n) return fail(BODEX_ERR_INVALID, "contact_link out of range");
    for (int a = 0; a < 3; ++a) H.clocal[i][a] = d->contact_local[3 * i + a];
    int chain[MAXJ], L = 0;
    for (int j = H.clink[i]; j >= 0; j = H.parent[j]) chain[L++] = j;
    if (L > MAXCHAIN) return fail(BODEX_ERR_INVALID, "contact chain longer than BODEX_MAX_CHAIN");
    H.chain_len[i] = L;
    for (int k = 0; k < L; ++k) {
      H.chain[i][k] = chain[L - 1 - k];
      H.jpos[i][chain[L - 1 - k]] = (int8_t)k;
    }
  }
  if (H.S < 0 || (H.S > 0 && !d->tip_samples)) return fail(BODEX_ERR_INVALID, "tip samples missing");
  bodex_hand_s* h = new bodex_hand_s();
  h->host = H;
  cudaError_t e = cudaMalloc(&h->dev, sizeof(HandDev));
  if (e != cudaSuccess) {
    delete h;
    return fail(BODEX_ERR_OOM, "cudaMalloc hand");
  }
  if (H.S > 0) {
    const size_t bytes = (size_t)m * H.S * 3 * sizeof(float);
    e = cudaMalloc(&h->tips, bytes);
    if (e != cudaSuccess) {
      cudaFree(h->dev);
      delete h;
      return fail(BODEX_ERR_OOM, "cudaMalloc tip samples");
    }
    e = cudaMemcpy(h->tips, d->tip_samples, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(h->tips);
      cudaFree(h->dev);
      delete h;
      return cuda_fail(e, "cudaMemcpy tip samples");
    }
  }
  e = cudaMemcpy(h->dev, &h->host, sizeof(HandDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (h->tips) cudaFree(h->tips);
    cudaFree(h->dev);
    delete h;
    return cuda_fail(e, "cudaMemcpy hand");
  }
  if (int r = upload_spheres(h, d)) {
    bodex_hand_destroy(h);
    return r;
  }
  *out = h;
  return BODEX_OK;
}

int bodex_hand_destroy(bodex_hand_t h) {
  if (!h) return BODEX_OK;
  if (h->tips) cudaFree(h->tips);
  if (h->coll_mem) cudaFree(h->coll_mem);
  cudaFree(h->dev);
  delete h;
  return BODEX_OK;
}

int bodex_object_create(const bodex_object_desc* d, void* stream, bodex_object_t* out) {
  if (!d || !out) return fail(BODEX_ERR_INVALID, "null argument");
  *out = nullptr;
  bodex_object_s* o = new bodex_object_s();
  std::memset(&o->dev, 0, sizeof(ObjDev));
  if (d->kind == 0) {
    if (!(d->radius > 0.f)) {
      delete o;
      return fail(BODEX_ERR_INVALID, "sphere radius must be > 0");
    }
    o->dev.kind = 0;
    o->dev.cx = d->center[0];
    o->dev.cy = d->center[1];
    o->dev.cz = d->center[2];
    o->dev.r = d->radius;
    o->dev.gcx = d->center[0];
    o->dev.gcy = d->center[1];
    o->dev.gcz = d->center[2];
  } else if (d->kind == 1) {
    const int N = d->n;
    if (N < 2 || !(d->h > 0.f) || !d->values) {
      delete o;
      return fail(BODEX_ERR_INVALID, "grid needs n >= 2, h > 0 and values");
    }
    const size_t cnt = (size_t)N * N * N;
    o->dev.kind = 1;
    o->dev.N = N;
    o->dev.h = d->h;
    o->dev.inv_h = 1.0f / d->h;
    o->dev.ox = d->origin[0];
    o->dev.oy = d->origin[1];
    o->dev.oz = d->origin[2];
    // gravity centre: mean of the node positions inside the object (double)
    double sx = 0, sy = 0, sz = 0;
    long long inside = 0;
    for (int iz = 0; iz < N; ++iz)
      for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix)
          if (d->values[((size_t)iz * N + iy) * N + ix] < 0.f) {
            sx += (double)d->origin[0] + (double)d->h * ix;
            sy += (double)d->origin[1] + (double)d->h * iy;
            sz += (double)d->origin[2] + (double)d->h * iz;
            ++inside;
          }
    if (inside > 0) {
      o->dev.gcx = (float)(sx / inside);
      o->dev.gcy = (float)(sy / inside);
      o->dev.gcz = (float)(sz / inside);
    } else {
      const double half = 0.5 * (double)d->h * (N - 1);
      o->dev.gcx = (float)(d->origin[0] + half);
      o->dev.gcy = (float)(d->origin[1] + half);
      o->dev.gcz = (float)(d->origin[2] + half);
    }
    cudaError_t e = cudaMalloc(&o->grid, cnt * sizeof(float));
    if (e != cudaSuccess) {
      delete o;
      return fail(BODEX_ERR_OOM, "cudaMalloc grid");
    }
    e = cudaMemcpyAsync(o->grid, d->values, cnt * sizeof(float), cudaMemcpyHostToDevice, as_stream(stream));
    if (e != cudaSuccess) {
      cudaFree(o->grid);
      delete o;
      return cuda_fail(e, "cudaMemcpyAsync grid");
    }
    o->dev.grid = o->grid;
  } else {
    delete o;
    return fail(BODEX_ERR_INVALID, "object kind must be 0 (sphere) or 1 (grid)");
  }
  *out = o;
  return BODEX_OK;
}

int bodex_object_destroy(bodex_object_t o) {
  if (!o) return BODEX_OK;
  if (o->grid) cudaFree(o->grid);
  delete o;
  return BODEX_OK;
}

int bodex_object_gravity_centre(bodex_object_t o, float out[3]) {
  if (!o || !out) return fail(BODEX_ERR_INVALID, "null argument");
  out[0] = o->dev.gcx;
  out[1] = o->dev.gcy;
  out[2] = o->dev.gcz;
  return BODEX_OK;
}

int bodex_fk_contacts(bodex_hand_t h, bodex_object_t o, const float* x, int B, float* c_w, float* p, float* n,
                      float* phi, float* G, int32_t* cell, int32_t* status, void* stream) {
  if (!h || !o || (!x && B > 0) || B < 0) return fail(BODEX_ERR_INVALID, "null handle/pose or B < 0");
  cudaStream_t st = as_stream(stream);
  switch (h->host.m) {
    case 3: return run_fk<3>(h, o, x, B, c_w, p, n, phi, G, cell, status, st);
    case 4: return run_fk<4>(h, o, x, B, c_w, p, n, phi, G, cell, status, st);
    case 5: return run_fk<5>(h, o, x, B, c_w, p, n, phi, G, cell, status, st);
  }
  return fail(BODEX_ERR_INVALID, "unsupported m");
}

int bodex_qp_solve_batch(const float* G, int B, int m, const float* T, int s, const bodex_qp_params* params,
                         float* y, float* z, float* lam, float* Q, int32_t* iters, int32_t* status, float* res,
                         void* stream) {
  if (B < 0 || s < 1 || s > SMAX) return fail(BODEX_ERR_INVALID, "B < 0 or s outside 1..16");
  if (B > 0 && (!G || !T || !y || !z || !lam || !Q)) return fail(BODEX_ERR_INVALID, "null array");
  if (int r = check_qp_params(params, m)) return r;
  if (params->strict && !status) return fail(BODEX_ERR_INVALID, "strict mode needs a status array");
  if (params->polish == 2 && !status) return fail(BODEX_ERR_INVALID, "polish = 2 needs a status array");
  AdmmCfg cfg = admm_cfg(*params);
  // K^-1 in FP64 for any residual target: an FP32 K^-1 raises the ADMM floor
  // (on the paper batch 98.2% instead of 99.5% of the QPs reach 1e-5)
  cfg.fp64_setup = params->eps_abs > 0.f ? 1 : 0;
  cudaStream_t st = as_stream(stream);
  if (m < 3 || m > 5) return fail(BODEX_ERR_INVALID, "m must be 3, 4 or 5");
  const int r = launch_qp(m, G, B, T, s, cfg, params->warm, y, z, lam, Q, iters, status, res, st);
  if (r || !params->strict || B == 0) return r;
  std::vector<int32_t> hs((size_t)B * s);
  BODEX_CUDA(cudaMemcpyAsync(hs.data(), status, hs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  BODEX_CUDA(cudaStreamSynchronize(st));
  for (int32_t v : hs)
    if (v & BODEX_ST_NOT_CONVERGED) return fail(BODEX_ERR_NOT_CONVERGED, "a QP missed eps_abs");
  return BODEX_OK;
}

int bodex_state_create(bodex_hand_t h, int B, int s, bodex_state_t* out) {
  if (!h || !out || B < 0 || s < 1 || s > SMAX) return fail(BODEX_ERR_INVALID, "bad state arguments");
  *out = nullptr;
  bodex_state_s* S = new bodex_state_s();
  S->B = B;
  S->s = s;
  S->m = h->host.m;
  S->D = h->host.D;
  const size_t nx = (size_t)B * S->D, ny = (size_t)B * s * 3 * S->m, nw = (size_t)B * s * (9 * S->m + 1);
  float** bufs[6] = {&S->x, &S->am, &S->av, &S->qy, &S->qw, &S->res};
  const size_t cnt[6] = {nx, nx, nx, ny, nw, (size_t)B};
  for (int k = 0; k < 6; ++k) {
    if (cnt[k] == 0) continue;
    if (cudaMalloc(bufs[k], cnt[k] * sizeof(float)) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaFree(*bufs[j]);
      delete S;
      return fail(BODEX_ERR_OOM, "cudaMalloc state");
    }
    cudaMemset(*bufs[k], 0, cnt[k] * sizeof(float));
  }
  if (cudaMalloc(&S->work, sizeof(int)) != cudaSuccess) {
    for (int k = 0; k < 6; ++k) cudaFree(*bufs[k]);
    delete S;
    return fail(BODEX_ERR_OOM, "cudaMalloc state");
  }
  *out = S;
  return BODEX_OK;
}

int bodex_state_destroy(bodex_state_t S) {
  if (!S) return BODEX_OK;
  cudaFree(S->work);
  cudaFree(S->res);
  cudaFree(S->x);
  cudaFree(S->am);
  cudaFree(S->av);
  cudaFree(S->qy);
  cudaFree(S->qw);
  delete S;
  return BODEX_OK;
}

int bodex_state_set_pose(bodex_state_t S, const float* x, void* stream) {
  if (!S || (!x && S->B > 0)) return fail(BODEX_ERR_INVALID, "null argument");
  if (S->B == 0) return BODEX_OK;
  cudaStream_t st = as_stream(stream);
  const size_t nx = (size_t)S->B * S->D;
  BODEX_CUDA(cudaMemcpyAsync(S->x, x, nx * sizeof(float), cudaMemcpyDeviceToDevice, st));
  BODEX_CUDA(cudaMemsetAsync(S->am, 0, nx * sizeof(float), st));
  BODEX_CUDA(cudaMemsetAsync(S->av, 0, nx * sizeof(float), st));
  BODEX_CUDA(cudaMemsetAsync(S->qy, 0, (size_t)S->B * S->s * 3 * S->m * sizeof(float), st));
  BODEX_CUDA(cudaMemsetAsync(S->qw, 0, (size_t)S->B * S->s * (9 * S->m + 1) * sizeof(float), st));
  S->t = 0;
  return BODEX_OK;
}

int bodex_state_get_pose(bodex_state_t S, float* x, void* stream) {
  if (!S || (!x && S->B > 0)) return fail(BODEX_ERR_INVALID, "null argument");
  if (S->B == 0) return BODEX_OK;
  BODEX_CUDA(cudaMemcpyAsync(x, S->x, (size_t)S->B * S->D * sizeof(float), cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
  return BODEX_OK;
}

int bodex_state_get_residual(bodex_state_t S, float* res, void* stream) {
  if (!S || (!res && S->B > 0)) return fail(BODEX_ERR_INVALID, "null argument");
  if (S->B == 0) return BODEX_OK;
  BODEX_CUDA(cudaMemcpyAsync(res, S->res, (size_t)S->B * sizeof(float), cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
  return BODEX_OK;
}

int bodex_state_get_adam(bodex_state_t S, float* m, float* v, int* step, void* stream) {
  if (!S) return fail(BODEX_ERR_INVALID, "null state");
  const size_t nx = (size_t)S->B * S->D * sizeof(float);
  if (m && nx) BODEX_CUDA(cudaMemcpyAsync(m, S->am, nx, cudaMemcpyDeviceToDevice, as_stream(stream)));
  if (v && nx) BODEX_CUDA(cudaMemcpyAsync(v, S->av, nx, cudaMemcpyDeviceToDevice, as_stream(stream)));
  if (step) *step = S->t;
  return BODEX_OK;
}

static int fill_args(FusedArgs& A, bodex_hand_t h, bodex_object_t o, const float* T, int s, int B,
                     const bodex_step_params* p) {
  if (!h || !o || !p || !T || s < 1 || s > SMAX || B < 0) return fail(BODEX_ERR_INVALID, "bad arguments");
  if (int r = check_qp_params(&p->qp, h->host.m)) return r;
  std::memset(&A, 0, sizeof(A));
  A.hand = h->dev;
  A.obj = o->dev;
  A.T = T;
  A.S = s;
  A.B = B;
  A.cfg = admm_cfg(p->qp);
  A.w_q = p->energy.w_q;
  A.w_d = p->energy.w_d;
  A.delta = p->energy.delta;
  A.lr_t = p->lr_t;
  A.lr_r = p->lr_r;
  A.b1 = p->b1;
  A.b2 = p->b2;
  A.adam_eps = p->adam_eps;
  // a tight residual target moves ADMM's fixed point with the backward
  // error of K^-1: build it in double there
  A.cfg.fp64_setup = (p->qp.eps_abs > 0.f && p->qp.eps_abs <= 2e-6f) ? 1 : 0;
  A.gpb = p->grasps_per_cta;
  if (p->energy.kind != BODEX_ENERGY_QP && p->energy.kind != BODEX_ENERGY_DFC)
    return fail(BODEX_ERR_INVALID, "energy.kind must be BODEX_ENERGY_QP or BODEX_ENERGY_DFC");
  A.dfc = p->energy.kind == BODEX_ENERGY_DFC;
  const bodex_energy_params& e = p->energy;
  if (!(e.eta_pen >= 0.f) || !(e.eta_lim >= 0.f)) return fail(BODEX_ERR_INVALID, "eta_pen and eta_lim must be >= 0");
  A.coll = (e.w_pen != 0.f || e.w_self != 0.f || e.w_lim != 0.f) ? 1 : 0;
  A.cd = h->coll;
  A.cp = CollParams{e.w_pen, e.w_self, e.w_lim, e.eta_pen, e.eta_lim};
  return BODEX_OK;
}

int bodex_energy_grad(bodex_hand_t h, bodex_object_t o, const float* x, int B, const float* T, int s,
                      const bodex_step_params* params, bodex_state_t warm, float* E, float* dEdx, float* Q,
                      float* y, int32_t* status, void* stream) {
  FusedArgs A;
  if (int r = fill_args(A, h, o, T, s, B, params)) return r;
  if (B > 0 && (!x || !E)) return fail(BODEX_ERR_INVALID, "null x or E");
  if (warm && (warm->B != B || warm->s != s || warm->m != h->host.m))
    return fail(BODEX_ERR_INVALID, "warm state shape mismatch");
  A.n_steps = 1;
  A.x_in = x;
  A.qy = warm ? warm->qy : nullptr;
  A.qw = warm ? warm->qw : nullptr;
  A.E = E;
  A.dEdx = dEdx;
  A.Qout = Q;
  A.yout = y;
  A.status = status;
  return dispatch_fused(h->host.m, MODE_EVAL, A, as_stream(stream));
}

int bodex_energy_adjoint(bodex_hand_t h, bodex_object_t o, const float* x, int B, const float* T, int s,
                         const bodex_step_params* params, const float* y, float* E, float* dEdx, int32_t* status,
                         void* stream) {
  FusedArgs A;
  if (int r = fill_args(A, h, o, T, s, B, params)) return r;
  if (B > 0 && (!x || !y || !dEdx)) return fail(BODEX_ERR_INVALID, "null x, y or dEdx");
  A.n_steps = 1;
  A.x_in = x;
  A.yin = y;
  A.E = E;
  A.dEdx = dEdx;
  A.status = status;
  return dispatch_fused(h->host.m, MODE_ADJOINT, A, as_stream(stream));
}

int bodex_step(bodex_hand_t h, bodex_object_t o, bodex_state_t S, const float* T, int s, int n_steps,
               const bodex_step_params* params, float* E_last, int32_t* status, void* stream) {
  if (!S) return fail(BODEX_ERR_INVALID, "null state");
  FusedArgs A;
  if (int r = fill_args(A, h, o, T, s, S->B, params)) return r;
  if (S->s != s || S->m != h->host.m) return fail(BODEX_ERR_INVALID, "state shape mismatch");
  if (n_steps < 0) return fail(BODEX_ERR_INVALID, "n_steps < 0");
  if (n_steps == 0) return BODEX_OK;
  A.n_steps = n_steps;
  A.t0 = S->t;
  A.x_state = S->x;
  A.am = S->am;
  A.av = S->av;
  A.qy = S->qy;
  A.qw = S->qw;
  A.E = E_last;
  A.status = status;
  A.res = S->res;
  const int r = dispatch_fused(h->host.m, MODE_STEP, A, as_stream(stream));
  if (r == BODEX_OK) S->t += n_steps;
  return r;
}

int bodex_step_multi(const bodex_job* jobs, int n_jobs, const bodex_step_params* params, void* stream) {
  if (n_jobs < 0 || n_jobs > BODEX_MAX_JOBS || (n_jobs > 0 && !jobs) || !params)
    return fail(BODEX_ERR_INVALID, "n_jobs must be 0..BODEX_MAX_JOBS with a job array");
  MultiArgs* MA = new MultiArgs();  // ~15 KB: kept off the host stack
  std::memset(MA, 0, sizeof(MultiArgs));
  size_t bytes = 0;
  int total = 0, nj = 0;
  int take[BODEX_MAX_JOBS], tiles[BODEX_MAX_JOBS];
  double cost[BODEX_MAX_JOBS];
  for (int j = 0; j < n_jobs; ++j) {
    const bodex_job& J = jobs[j];
    bodex_state_t S = J.state;
    if (!J.hand || !J.obj || !S) {
      delete MA;
      return fail(BODEX_ERR_INVALID, "job with a null handle");
    }
    if (S->s != J.s || S->m != J.hand->host.m || S->D != J.hand->host.D || J.n_steps < 0) {
      delete MA;
      return fail(BODEX_ERR_INVALID, "job state shape mismatch or n_steps < 0");
    }
    if (S->B == 0 || J.n_steps == 0) continue;
    FusedArgs& A = MA->job[nj];
    if (int r = fill_args(A, J.hand, J.obj, J.T, J.s, S->B, params)) {
      delete MA;
      return r;
    }
    const int m = J.hand->host.m;
    int gpb = 0;
    size_t b = 0;
    switch (m) {
      case 3: gpb = pick_gpb<3>(J.s, A.gpb); b = Lay<3>::bytes(gpb); break;
      case 4: gpb = pick_gpb<4>(J.s, A.gpb); b = Lay<4>::bytes(gpb); break;
      default: gpb = pick_gpb<5>(J.s, A.gpb); b = Lay<5>::bytes(gpb); break;
    }
    A.gpb = gpb;
    A.n_steps = J.n_steps;
    A.t0 = S->t;
    A.x_state = S->x;
    A.am = S->am;
    A.av = S->av;
    A.qy = S->qy;
    A.qw = S->qw;
    A.E = J.E_last;
    A.status = J.status;
    A.res = S->res;
    MA->m[nj] = m;
    tiles[nj] = (S->B + gpb - 1) / gpb;
    // cost of one tile: steps x wrenches x (ADMM work per iteration, 26 m + 9 m^2 + ...,
    // taken as m^2; or m for the exact solve, whose oracle is linear in m)
    const bool ex = params->qp.solver == BODEX_QP_EXACT;
    cost[nj] = (double)J.n_steps * J.s * (ex ? m : m * m);
    total += tiles[nj];
    bytes = std::max(bytes, b);
    take[nj] = j;
    ++nj;
  }
  MA->n_jobs = nj;
  MA->total = total;
  int r = BODEX_OK;
  if (nj > 0) {
    // work items job by job: the costliest job's tiles first (stable on
    // ties) for the pulling schedule, the caller's order otherwise
    const bool pull = params->work_pulling != 0;
    int ord[BODEX_MAX_JOBS];
    for (int k = 0; k < nj; ++k) ord[k] = k;
    if (pull) std::stable_sort(ord, ord + nj, [&](int a, int b2) { return cost[a] > cost[b2]; });
    int acc = 0;
    for (int k = 0; k < nj; ++k) {
      MA->order_job[k] = ord[k];
      MA->order_begin[k] = acc;
      acc += tiles[ord[k]];
    }
    MA->order_begin[nj] = acc;
    // the item counter lives with the first job's state (calls that share a
    // state are serialised by the caller, so no two launches share it)
    MA->counter = jobs[take[0]].state->work;
    cudaStream_t st = as_stream(stream);
    if (pull) {
      const cudaError_t e = cudaMemsetAsync(MA->counter, 0, sizeof(int), st);
      if (e != cudaSuccess) {
        delete MA;
        return cuda_fail(e, "cudaMemsetAsync(work counter)");
      }
    }
    const bool exact = params->qp.solver == BODEX_QP_EXACT;
    const bool adapt = !exact && params->qp.eps_abs > 0.f && params->qp.adaptive_rho;
    r = launch_multi(adapt, exact, pull, *MA, bytes, st);
    if (r == BODEX_OK)
      for (int k = 0; k < nj; ++k) jobs[take[k]].state->t += jobs[take[k]].n_steps;
  }
  delete MA;
  return r;
}

// ============================================================================ refinement ABI
extern "C" int bodex_refine(bodex_hand_t h, bodex_object_t o, bodex_state_t S, const float* p_coarse, int n_steps,
                            float delta, float w_qp, const bodex_step_params* p, float* E_last, int32_t* kstar,
                            int32_t* status, void* stream) {
  if (!h || !o || !S || !p) return fail(BODEX_ERR_INVALID, "null argument");
  if (h->host.S <= 0 || !h->tips) return fail(BODEX_ERR_INVALID, "hand has no fingertip samples");
  if (S->m != h->host.m || S->D != h->host.D) return fail(BODEX_ERR_INVALID, "state shape mismatch");
  if (n_steps < 0) return fail(BODEX_ERR_INVALID, "n_steps < 0");
  if (S->B > 0 && !p_coarse) return fail(BODEX_ERR_INVALID, "null p_coarse");
  if (n_steps == 0 || S->B == 0) return BODEX_OK;
  RefineArgs A;
  std::memset(&A, 0, sizeof(A));
  A.hand = h->dev;
  A.tips = h->tips;
  A.obj = o->dev;
  A.B = S->B;
  A.pc = p_coarse;
  A.delta = delta;
  A.w_d = p->energy.w_d;
  A.w_qp = w_qp;
  A.lr_t = p->lr_t;
  A.lr_r = p->lr_r;
  A.b1 = p->b1;
  A.b2 = p->b2;
  A.adam_eps = p->adam_eps;
  A.n_steps = n_steps;
  A.t0 = S->t;
  A.x = S->x;
  A.am = S->am;
  A.av = S->av;
  A.E = E_last;
  A.kstar = kstar;
  A.status = status;
  int r;
  switch (h->host.m) {
    case 3: r = run_refine<3>(A, as_stream(stream)); break;
    case 4: r = run_refine<4>(A, as_stream(stream)); break;
    case 5: r = run_refine<5>(A, as_stream(stream)); break;
    default: return fail(BODEX_ERR_INVALID, "unsupported m");
  }
  if (r == BODEX_OK) S->t += n_steps;
  return r;
}

extern "C" int bodex_contact_metrics(bodex_hand_t h, bodex_object_t o, const float* x, int B, float* d, float* cdc,
                                     void* stream) {
  if (!h || !o) return fail(BODEX_ERR_INVALID, "null handle");
  if (B < 0) return fail(BODEX_ERR_INVALID, "B < 0");
  if (B > 0 && (!x || !d)) return fail(BODEX_ERR_INVALID, "null x or d");
  if (B == 0) return BODEX_OK;
  MetricsArgs A;
  std::memset(&A, 0, sizeof(A));
  A.hand = h->dev;
  A.tips = (h->host.S > 0) ? h->tips : nullptr;
  A.obj = o->dev;
  A.B = B;
  A.x = x;
  A.d = d;
  A.cdc = cdc;
  switch (h->host.m) {
    case 3: return run_metrics<3>(A, as_stream(stream));
    case 4: return run_metrics<4>(A, as_stream(stream));
    case 5: return run_metrics<5>(A, as_stream(stream));
    default: return fail(BODEX_ERR_INVALID, "unsupported m");
  }
}

// ============================================================================ squeeze pose
// x_s = 2 x - x_p (Sec. IV-D), elementwise over B * D floats; 2 x is exact
// in float, so the one rounding gives the same value as the formula.
__global__ void __launch_bounds__(256) squeeze_kernel(const float* __restrict__ x, const float* __restrict__ xp,
                                                      size_t n, float* __restrict__ xs) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    xs[i] = fmaf(2.f, x[i], -xp[i]);
}

extern "C" int bodex_squeeze_pose(const float* x, const float* x_p, int B, int D, float* x_s, void* stream) {
  if (B < 0 || D < 1) return fail(BODEX_ERR_INVALID, "B < 0 or D < 1");
  if (B > 0 && (!x || !x_p || !x_s)) return fail(BODEX_ERR_INVALID, "null array");
  if (B == 0) return BODEX_OK;
  const size_t n = (size_t)B * D;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
  (void)cudaGetLastError();
  squeeze_kernel<<<blocks, 256, 0, as_stream(stream)>>>(x, x_p, n, x_s);
  return launch_err("squeeze_kernel launch");
}

// ============================================================================ allocation-free step
// Some callers cannot allocate device memory once they are running: a robot
// controller that reserves everything at start-up so that its control loop
// has bounded latency, an application whose memory pool owns the whole
// device and forbids cudaMalloc, or a plug-in hosted by such a process.
// bodex_step_noalloc serves them.  The per-grasp state that bodex_step keeps
// in a bodex_state_t (Adam moments and the ADMM warm start of every QP) lives
// instead in the fixed array below, which every GPU that loads this library
// holds until the process exits.  The caller still passes the poses, the
// wrenches and the outputs.
namespace {
constexpr size_t kNoallocScratchFloats = size_t(1) << 20;  // 4 MiB per device
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_addr[kNoallocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[kNoallocScratchFloats];

// Device address of the scratch array on the current device.  Host code may
// not use the symbol itself (it names a host-side stand-in), so the address
// is looked up once per device, with that device current, and cached.
static int noalloc_scratch(float** out) {
  int dev = 0;
  BODEX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(BODEX_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_addr[dev];
  return BODEX_OK;
}

extern "C" int bodex_step_noalloc(bodex_hand_t h, bodex_object_t o, float* x, int B, const float* T, int s,
                                  int n_steps, const bodex_step_params* params, float* E_last, int32_t* status,
                                  void* stream) {
  FusedArgs A;
  if (int r = fill_args(A, h, o, T, s, B, params)) return r;
  if (B > 0 && !x) return fail(BODEX_ERR_INVALID, "null x");
  if (n_steps < 0) return fail(BODEX_ERR_INVALID, "n_steps < 0");
  const size_t D = (size_t)h->host.D, m = (size_t)h->host.m;
  auto up = [](size_t v) { return (v + 63) & ~size_t(63); };  // 256-byte aligned regions
  const size_t nA = up((size_t)B * D), nY = up((size_t)B * s * 3 * m), nW = up((size_t)B * s * (9 * m + 1));
  const size_t need = 2 * nA + nY + nW;
  if (need > kNoallocScratchFloats)
    return fail(BODEX_ERR_INVALID,
                "bodex_step_noalloc: B * (2 (6+n) + s (12 m + 1)) floats exceed its fixed 4 MiB scratch "
                "(1048576 floats); use bodex_state_create + bodex_step for larger batches");
  if (n_steps == 0 || B == 0) return BODEX_OK;
  float* base = nullptr;
  if (int r = noalloc_scratch(&base)) return r;
  cudaStream_t st = as_stream(stream);
  // the array keeps the previous call's contents: Adam moments and warm
  // starts must start at zero
  BODEX_CUDA(cudaMemsetAsync(base, 0, need * sizeof(float), st));
  A.n_steps = n_steps;
  A.t0 = 0;
  A.x_state = x;
  A.am = base;
  A.av = base + nA;
  A.qy = base + 2 * nA;
  A.qw = base + 2 * nA + nY;
  A.E = E_last;
  A.status = status;
  return dispatch_fused((int)m, MODE_STEP, A, st);
}

}  // extern "C"
