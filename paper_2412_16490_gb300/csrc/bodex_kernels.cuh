// Kernels and launch helpers shared by the library's translation units:
// the per-grasp shared-memory layout, the batched-QP kernel, the fused
// step kernel and the several-job kernel.  bodex.cu holds the C ABI and the
// small kernels; qp.cu, fused_m3.cu, fused_m4.cu, fused_m5.cu and
// fused_multi.cu instantiate the heavy kernels, so that nvcc compiles them
// in parallel.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <mutex>
#include <string>

#include "../../include/bodex.h"
#include "bodex_device.cuh"

namespace bodex {
// error state of the C ABI (bodex.cu)
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int launch_err(const char* what);
}  // namespace bodex

using namespace bodex;

// ============================================================================ shared-memory layout
constexpr int CTA_LANES = 96;

__host__ __device__ constexpr int align4(int v) { return (v + 3) & ~3; }

template <int M>
struct Lay {
  static constexpr int NV = 3 * M, NC = 9 * M + 1, NVP = (NV + 3) & ~3;
  // K^-1 block per grasp (packed upper triangle in whole float4s); the
  // stride is skewed (== 20 mod 32 words) so that lanes of two or three
  // grasps in one warp hit disjoint banks.
  static constexpr int KT = 4 * Admm<M>::NTRI4;
  static constexpr int KS = KT + ((20 - KT % 32) + 32) % 32;
  static constexpr int CTW = 24;  // floats per contact record
  static constexpr int oG = 0;
  static constexpr int oK = align4(oG + 6 * NV);  // K^-1 setup scratch (16-byte aligned)
  static constexpr int oCT = oK + WoodburyScratch<M, double>::floats;
  // per-lane record of the QP outputs: r_j (6; read as a float4 and a
  // float2 by the dE/dG reduction, so records start on 16-byte boundaries),
  // two pad words, then y_j
  static constexpr int RYW = 8 + NVP;
  static constexpr int oRY = oCT + CTW * M;
  static constexpr int oQ = oRY + SMAX * RYW;
  static constexpr int oDG = oQ + SMAX;
  static constexpr int oCB = oDG + 6 * NV;
  static constexpr int oX = oCB + M * (6 + MAXCHAIN);
  static constexpr int oAM = oX + MAXD;
  static constexpr int oAV = oAM + MAXD;
  static constexpr int oJW = oAV + MAXD;  // chain joint axes/points, M x MAXCHAIN x 6
  static constexpr int oGC = oJW + M * MAXCHAIN * 6;  // collision gradient [MAXD], energy by lane [SMAX]
  static constexpr int oSC = oGC + MAXD + SMAX;
  // collision scratch: link frames in the K^-1 setup scratch, sphere centres
  // and slot sums in the r / Q / dE/dG block (both dead before A4)
  static constexpr int COLL_FR = WoodburyScratch<M, double>::floats;
  static constexpr int COLL_CS = SMAX * RYW + SMAX + 6 * NV;
  // per-grasp stride == 12 (mod 32) words: the two or three grasps that
  // share a warp then map the same offset to different banks
  static constexpr int PER = align4(oSC + 4) + ((12 - align4(oSC + 4) % 32) + 32) % 32;
  static constexpr int HAND_WORDS = align4((int)(sizeof(HandDev) / 4));
  static size_t bytes(int gpb) { return 4u * (size_t)(HAND_WORDS + gpb * (KS + PER)); }
};

// Contact record in shared memory: c(3) p(3) n(3) phi g(3) h(6) cell(3) degenerate.
__device__ __forceinline__ void store_ct(float* r, const ContactGeo& k) {
  for (int a = 0; a < 3; ++a) {
    r[a] = k.c[a];
    r[3 + a] = k.p[a];
    r[6 + a] = k.n[a];
    r[10 + a] = k.g[a];
    r[19 + a] = __int_as_float(k.cell[a]);
  }
  r[9] = k.phi;
  for (int e = 0; e < 6; ++e) r[13 + e] = k.h[e];
  r[22] = __int_as_float(k.degenerate);
}
__device__ __forceinline__ ContactGeo load_ct(const float* r) {
  ContactGeo k;
  for (int a = 0; a < 3; ++a) {
    k.c[a] = r[a];
    k.p[a] = r[3 + a];
    k.n[a] = r[6 + a];
    k.g[a] = r[10 + a];
    k.cell[a] = __float_as_int(r[19 + a]);
  }
  k.phi = r[9];
  for (int e = 0; e < 6; ++e) k.h[e] = r[13 + e];
  k.degenerate = __float_as_int(r[22]);
  return k;
}

__device__ __forceinline__ void copy_hand_to_smem(const HandDev* src, float* dst) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  const int words = (int)(sizeof(HandDev) / 4);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = __ldg(s + i);
}

__device__ __forceinline__ bool finite3(const float* v) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

// ============================================================================ per-grasp QP setup (shared by kernels)
// K^-1 of every grasp of the CTA (Woodbury form, all lanes); must be called
// by every thread of the CTA (contains barriers).
// Double precision when the host asks for it (solves that iterate to a
// tight residual target), single precision otherwise; the branch is
// uniform per launch.
template <int M, bool UNROLL = false>
__device__ inline void setup_kinv(bool active, int lane, int S, const float* Gs, float* scratch, float* Kinv,
                                  const AdmmCfg& cfg) {
  if (cfg.fp64_setup) setup_kinv_woodbury<M, double>(active, lane, S, Gs, scratch, Kinv, cfg);
  else setup_kinv_woodbury<M, float, UNROLL>(active, lane, S, Gs, scratch, Kinv, cfg);
}

// ============================================================================ kernel: batched QP
// One QP per thread, the grasps' K^-1 shared by their QPs.  QPs converge
// after very different iteration counts (at 1e-5 on the paper geometry the
// median is 400, the slowest of a warp's 32 about 3100), and a warp runs
// until its last QP stops.  So at every residual check the QPs still running
// are repacked, through shared memory, into the lowest warps of the CTA: a
// warp whose QPs all stopped waits at the barrier and issues nothing while
// the others iterate.  A QP carries its iterate, -q, its iteration count and
// its slot (grasp, wrench); K^-1, G and rho stay with the grasp.
// The last QPs of a CTA (at most 32 / m) run in a wide form on warp 0: one
// QP per m lanes, lane i holding contact i's rows, the rhs exchanged by warp
// shuffles and each lane forming three rows of alpha K^-1 rhs from a dense
// copy of the grasp's K^-1; the residual check is spread over the lanes
// too.  Alone on its SM, a QP's iteration is bound by its chain of dependent
// instructions, which the wide form shortens: the slowest QPs of a batch
// finish sooner (the paper batch: 2.64 ms instead of 3.26 ms).  Every
// multiply-add is the one-lane form's, in the same order (row r of the
// product sums j = 0 .. nv-1 in both), so the iterates agree bitwise.
//
// Shared memory: alpha K^-1 per grasp (stride as in the fused kernel), the
// per-grasp block (G, Woodbury scratch, votes, rho), the parking area (one
// record per QP) and one count per warp.
template <int M, int CONE>
struct LayQP {
  static constexpr int NV = 3 * M, NC = CONE == CONE_SOC ? 4 * M + 1 : 9 * M + 1;
  static constexpr int KS = Lay<M>::KS;
  static constexpr int oG = 0;
  static constexpr int oK = align4(6 * NV);  // Woodbury scratch (16-byte aligned)
  static constexpr int oVote = oK + WoodburyScratch<M, double>::floats;
  static constexpr int oRho = oVote + SMAX;  // the grasp's rho; oRho + 1: its rho before the last vote
  static constexpr int PER0 = align4(oRho + 2);
  static constexpr int PER = PER0 + ((12 - PER0 % 32) + 32) % 32;
  // parked QP: y, w, -q, then (iterations, slot); an odd count of float4s
  // per record keeps eight consecutive records on distinct banks
  static constexpr int pW = align4(NV), pM = pW + align4(NC), pI = pM + align4(NV);
  static constexpr int PW0 = pI + 4;
  static constexpr int PW = (PW0 / 4) % 2 ? PW0 : PW0 + 4;
  // wide form: QPs per warp, w rows per contact, dense K^-1 row stride
  // (the dense row stride is an odd number of float4s, so that the lanes of
  // a quarter-warp, which read different rows, hit distinct bank groups)
  static constexpr int QPW = 32 / M, WPC = CONE == CONE_SOC ? 4 : 9;
  static constexpr int NVP = (align4(NV) / 4) % 2 ? align4(NV) : align4(NV) + 4;
  static constexpr int WIDE_PER_QP = PW + NV * NVP;  // a record and a dense K^-1 per wide QP
  static size_t bytes(int gpb, int s) { return 4u * ((size_t)gpb * (KS + PER) + (size_t)gpb * s * PW + 32); }
};

template <int M, int CONE>
__global__ void __launch_bounds__(CTA_LANES, 4) qp_solve_kernel(const float* __restrict__ Gin, int B,
                                                                const float* __restrict__ T, int S, AdmmCfg cfg,
                                                                int warm, float* yio, float* zio, float* lio,
                                                                float* Qout, int32_t* iters_out, int32_t* status_out,
                                                                float* res_out) {
  using L = LayQP<M, CONE>;
  constexpr int NV = L::NV, NC = L::NC;
  extern __shared__ __align__(16) float smem[];
  const int GPB = blockDim.x / S;
  // setup role of this thread: lane `lane` of grasp gl of the CTA
  const int gl = threadIdx.x / S, lane = threadIdx.x % S;
  const bool role = (gl < GPB) && (blockIdx.x * GPB + gl < B);
  float* const park = smem + GPB * (L::KS + L::PER);
  int* const wcount = reinterpret_cast<int*>(park + GPB * S * L::PW);
  auto kin = [&](int g) { return smem + g * L::KS; };
  auto per = [&](int g) { return smem + GPB * L::KS + g * L::PER; };
  if (role) {
    const size_t b = (size_t)blockIdx.x * GPB + gl;
    for (int e = lane; e < 6 * NV; e += S) per(gl)[L::oG + e] = Gin[b * 6 * NV + e];
    if (lane == 0) per(gl)[L::oRho] = per(gl)[L::oRho + 1] = cfg.rho;
  }
  __syncthreads();
  setup_kinv<M>(role, lane, S, per(gl) + L::oG, per(gl) + L::oK, kin(gl), cfg);
  const bool adaptive = cfg.eps > 0.f && cfg.adapt;  // uniform
  const int check = cfg.eps > 0.f ? cfg.check : cfg.iters;  // without a target: residuals once, at the end
  const size_t q0 = (size_t)blockIdx.x * GPB * S;         // first QP of the CTA
  // the QP this thread runs: slot p = g * S + j of the CTA (at first its own), -1 for none
  int p = role ? (int)threadIdx.x : -1;
  int it = 0;
  float y[NV], w[NC], mq[NV];
  if (p >= 0) {
    float t[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) t[r] = T[lane * 6 + r];
    neg_q<M>(per(gl) + L::oG, t, cfg.beta, mq);
    const size_t q = q0 + p;
    if (warm) {
#pragma unroll
      for (int a = 0; a < NV; ++a) y[a] = yio[q * NV + a];
#pragma unroll
      for (int r = 0; r < NC; ++r) w[r] = zio[q * NC + r] + lio[q * NC + r] / cfg.rho;
    } else {
#pragma unroll
      for (int a = 0; a < NV; ++a) y[a] = 0.f;
#pragma unroll
      for (int r = 0; r < NC; ++r) w[r] = 0.f;
    }
  }
  // y, z = Pi(w), lam = rho (w - Pi(w)), Q, iterations, residuals and status of slot pp
  auto finish = [&](int pp, float rp, float rd, bool conv) {
    const int g = pp / S, j = pp % S;
    const size_t q = q0 + pp;
    const float* Gg = per(g) + L::oG;
    const float rho = per(g)[L::oRho];
    float Q = 0.f;
    bool fin = true;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      float s = cfg.beta * T[j * 6 + r];
#pragma unroll
      for (int a = 0; a < NV; ++a) s = fmaf(-Gg[r * NV + a], y[a], s);
      Q = fmaf(s, s, Q);
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      yio[q * NV + a] = y[a];
      fin = fin && isfinite(y[a]);
      Q = fmaf(cfg.eps_reg * y[a], y[a], Q);  // regularised value when eps_reg > 0
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      const float pr = CONE == CONE_SOC ? proj_row_soc<M>(w, r, cfg.gamma) : proj_row<M>(w[r], r, cfg.gamma);
      zio[q * NC + r] = pr;
      lio[q * NC + r] = rho * (w[r] - pr);
    }
    Qout[q] = Q;
    if (iters_out) iters_out[q] = it;
    if (res_out) {
      res_out[2 * q] = rp;
      res_out[2 * q + 1] = rd;
    }
    int st = 0;
    if (!fin || !isfinite(Q)) st |= BODEX_ST_NONFINITE;
    if (cfg.eps > 0.f && !conv) st |= BODEX_ST_NOT_CONVERGED;
    if (status_out) status_out[q] = st;
  };
  // parking record r: the iterate, -q, the iteration count and the slot
  auto park_store = [&](int r) {
    float* rec = park + r * L::PW;
#pragma unroll
    for (int a = 0; a < NV; ++a) rec[a] = y[a];
#pragma unroll
    for (int k = 0; k < NC; ++k) rec[L::pW + k] = w[k];
#pragma unroll
    for (int a = 0; a < NV; ++a) rec[L::pM + a] = mq[a];
    reinterpret_cast<int*>(rec)[L::pI] = it;
    reinterpret_cast<int*>(rec)[L::pI + 1] = p;
  };
  auto park_load = [&](int r) {
    const float* rec = park + r * L::PW;
#pragma unroll
    for (int a = 0; a < NV; ++a) y[a] = rec[a];
#pragma unroll
    for (int k = 0; k < NC; ++k) w[k] = rec[L::pW + k];
#pragma unroll
    for (int a = 0; a < NV; ++a) mq[a] = rec[L::pM + a];
    it = reinterpret_cast<const int*>(rec)[L::pI];
    p = reinterpret_cast<const int*>(rec)[L::pI + 1];
  };
  // adaptive rho, one decision per grasp (lane 0 of its setup role): rho
  // moves by the geometric mean of its running QPs' proposals when that is
  // more than 5x (clamped to [1e-6, 1e6]); returns whether it moved
  auto decide = [&]() -> bool {
    if (!(role && lane == 0)) return false;
    float* pg = per(gl);
    float sh = 0.f;
    int cnt = 0;
    for (int j = 0; j < S; ++j) {
      const float v = pg[L::oVote + j];
      sh += v;
      cnt += v != 0.f;
    }
    const float cur = pg[L::oRho];
    float nxt = cur;
    if (cnt > 0 && fabsf(sh / cnt) > 1.6094379f)  // log 5
      nxt = fminf(fmaxf(cur * __expf(sh / cnt), 1e-6f), 1e6f);
    pg[L::oRho + 1] = cur;
    pg[L::oRho] = nxt;
    return nxt != cur;
  };
  // K^-1 of the grasps whose rho moved (every thread; barriers inside)
  auto rebuild = [&]() {
    AdmmCfg cl = cfg;
    bool upd = false;
    if (role) {
      cl.rho = per(gl)[L::oRho];
      upd = cl.rho != per(gl)[L::oRho + 1];
    }
    setup_kinv<M>(upd, lane, S, per(gl) + L::oG, per(gl) + L::oK, kin(gl), cl);
  };
  const int warp = threadIdx.x / 32, wl = threadIdx.x % 32;
  const int nw = min(32, (int)blockDim.x - 32 * warp);
  const unsigned wmask = nw == 32 ? 0xffffffffu : (1u << nw) - 1u;  // this warp's threads
  int warps = (blockDim.x + 31) / 32;                                  // warps that hold running QPs
  // warps that take wide groups: warp 0 when it is full and the parking area
  // has room.  (Groups in every full warp, up to 18 QPs at m = 5, took
  // 3.05 ms on the paper batch against 2.68 ms for warp 0 alone: the SMs
  // turn issue-bound again.)
  const int wide_warps = (blockDim.x >= 32 && GPB * S * L::PW >= L::QPW * L::WIDE_PER_QP) ? 1 : 0;
  const bool wide_ok = cfg.eps > 0.f && wide_warps > 0;
  int n_run;
#pragma unroll 1
  for (;;) {
    bool run = p >= 0;
    if (run) {
      const int g = p / S;
      const float rho = per(g)[L::oRho];
      const float* kg = kin(g);
      const float* Gg = per(g) + L::oG;
      const int chunk = min(check, cfg.iters - it);
#pragma unroll 1
      for (int k = 0; k < chunk; ++k) {
        if (CONE == CONE_SOC) admm_iteration_soc<M>(y, w, mq, kg, cfg, rho);
        else admm_iteration<M>(y, w, mq, kg, cfg, rho);
      }
      it += chunk;
      // residuals from the parked copy: computed from registers, they would
      // need more than the 168 a thread has next to the iterate
      float rp, rd, scale[2];
      park_store(threadIdx.x);
      {
        const float* rec = park + threadIdx.x * L::PW;
        if (CONE == CONE_SOC) admm_residuals_soc<M, true>(rec, rec + L::pW, rec + L::pM, Gg, cfg, rho, rp, rd, scale);
        else admm_residuals<M, true>(rec, rec + L::pW, rec + L::pM, Gg, cfg, rho, rp, rd, scale);
      }
      park_load(threadIdx.x);
      const bool conv = cfg.eps > 0.f && rp <= cfg.eps && rd <= cfg.eps;
      if (conv || it >= cfg.iters) {
        finish(p, rp, rd, conv);
        run = false;
      }
      // residual balancing (OSQP, Stellato et al. 2020, Sec. 5.2): each
      // running QP proposes rho_vote (normalised residuals) for its grasp; 0 once stopped
      if (adaptive) per(g)[L::oVote + p % S] = run ? rho_vote(rp, rd, scale) : 0.f;
      if (!run) p = -1;
    }
    n_run = __syncthreads_count(run);
    if (n_run == 0) break;
    if (adaptive) {
      if (!__syncthreads_or(decide())) goto repack;  // no grasp of the CTA changed rho
      const bool mine = p >= 0;
      if (mine) {  // re-express the iterate at the grasp's new rho, then park it (its registers go to the setup)
        const float* pg = per(p / S);
        if (pg[L::oRho] != pg[L::oRho + 1]) rescale_w<M, CONE>(w, pg[L::oRho + 1] / pg[L::oRho], cfg);
        park_store(threadIdx.x);
      }
      rebuild();
      if (mine) park_load(threadIdx.x);
    }
  repack:
    if (wide_ok && n_run <= wide_warps * L::QPW) {
      // to the wide form: the running QPs parked in thread order (record r)
      const unsigned bal = __ballot_sync(wmask, p >= 0);
      if (wl == 0) wcount[warp] = __popc(bal);
      __syncthreads();
      if (p >= 0) {
        int r = __popc(bal & ((1u << wl) - 1u));
        for (int k = 0; k < warp; ++k) r += wcount[k];
        park_store(r);
      }
      __syncthreads();
      break;
    }
    if ((n_run + 31) / 32 < warps) {
      // repack: running QPs, in thread order, to threads 0 .. n_run - 1
      const unsigned bal = __ballot_sync(wmask, p >= 0);
      if (wl == 0) wcount[warp] = __popc(bal);
      __syncthreads();
      if (p >= 0) {
        int r = __popc(bal & ((1u << wl) - 1u));
        for (int k = 0; k < warp; ++k) r += wcount[k];
        park_store(r);
      }
      __syncthreads();
      p = -1;
      if ((int)threadIdx.x < n_run) park_load(threadIdx.x);
      warps = (n_run + 31) / 32;
    }
  }
  if (n_run == 0) return;
  // wide form (see above): group gi (QPW per wide warp) takes record gi,
  // its lane ci the rows of contact ci and a dense copy of rows 3ci .. 3ci+2
  // of the grasp's alpha K^-1 (in the parking area, after the records)
  constexpr int WPC = L::WPC, NVP = L::NVP;
  const int ci = wl % M, gb = (wl / M) * M;  // contact; first lane of the group in the warp
  const bool in_group = wl < L::QPW * M;     // lanes past the last whole group stay idle
  const int gi = warp * L::QPW + (in_group ? wl / M : 0);
  float wy[3] = {0.f, 0.f, 0.f}, ww[WPC], wmq[3] = {0.f, 0.f, 0.f}, wsum = 0.f;
#pragma unroll
  for (int k = 0; k < WPC; ++k) ww[k] = 0.f;
  float* Kd = park;  // any valid address for an idle lane
  p = -1;
  const bool wide_warp = warp < wide_warps;
  if (wide_warp && in_group && gi < n_run) {
    const float* rec = park + gi * L::PW;
    it = reinterpret_cast<const int*>(rec)[L::pI];
    p = reinterpret_cast<const int*>(rec)[L::pI + 1];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      wy[r] = rec[3 * ci + r];
      wmq[r] = rec[L::pM + 3 * ci + r];
    }
#pragma unroll
    for (int k = 0; k < WPC; ++k) ww[k] = rec[L::pW + WPC * ci + k];
    wsum = rec[L::pW + NC - 1];
    Kd = park + wide_warps * L::QPW * L::PW + gi * (NV * NVP) + 3 * ci * NVP;
  }
  // rows 3ci .. 3ci+2 of the grasp's alpha K^-1, dense (this lane's own rows)
  auto copy_rows = [&]() {
    const float* kg = kin(p / S);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int j = 0; j < NVP; ++j) {
        const int a = min(3 * ci + r, j), b = max(3 * ci + r, j);
        Kd[r * NVP + j] = j < NV ? kg[Admm<M>::tri(a, b)] : 0.f;
      }
  };
  if (p >= 0) copy_rows();
#pragma unroll 1
  for (;;) {
    bool run = false;
    if (wide_warp) {
      const bool mine = p >= 0;
      const int g = mine ? p / S : 0;
      const float rho = per(g)[L::oRho];
      // running QPs advance in lockstep rounds, so they share `it`
      const int chunk = __reduce_max_sync(0xffffffffu, mine ? min(check, cfg.iters - it) : 0);
      const float al = cfg.alpha, bl = 1.0f - cfg.alpha;
#pragma unroll 1
      for (int k = 0; k < chunk; ++k) {
        const float vsum = fmaf(2.f, fmaxf(wsum, cfg.gamma), -wsum);
        float rhs3[3], pc3[3];
        if (CONE == CONE_SOC) soc_contact_rhs(ww, vsum, wy, wmq, cfg, rho, rhs3, pc3);
        else pyr_contact_rhs(ww, vsum, wy, wmq, cfg, rho, rhs3);
        float ra[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) ra[j] = __shfl_sync(0xffffffffu, rhs3[j % 3], gb + j / 3);
        float yt3[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const float4* row = reinterpret_cast<const float4*>(Kd + r * NVP);
          float acc = 0.f;
#pragma unroll
          for (int j4 = 0; j4 < NVP / 4; ++j4) {
            const float4 kv = row[j4];
            if (4 * j4 + 0 < NV) acc = fmaf(kv.x, ra[4 * j4 + 0], acc);
            if (4 * j4 + 1 < NV) acc = fmaf(kv.y, ra[4 * j4 + 1], acc);
            if (4 * j4 + 2 < NV) acc = fmaf(kv.z, ra[4 * j4 + 2], acc);
            if (4 * j4 + 3 < NV) acc = fmaf(kv.w, ra[4 * j4 + 3], acc);
          }
          yt3[r] = acc;
        }
        float sumn = 0.f;
#pragma unroll
        for (int i = 0; i < M; ++i) sumn += __shfl_sync(0xffffffffu, yt3[0], gb + i);
        if (CONE == CONE_SOC) soc_contact_update(ww, pc3, yt3[0], yt3[1], yt3[2], cfg);
        else pyr_contact_update(ww, yt3[0], yt3[1], yt3[2], cfg);
        wsum = fmaf(-al, fmaxf(wsum, cfg.gamma), wsum + sumn);
#pragma unroll
        for (int r = 0; r < 3; ++r) wy[r] = fmaf(bl, wy[r], yt3[r]);
      }
      it += chunk;
      // residuals, spread over the group: every lane gathers y and forms
      // G y, then its contact's primal rows and dual components; the group
      // takes the maxima (the one-lane function's values, bitwise)
      float ya[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) ya[j] = __shfl_sync(0xffffffffu, wy[j % 3], gb + j / 3);
      const float* Gg = per(g) + L::oG;
      float sumn = 0.f, rp = 0.f, rd = 0.f, np = 0.f, nd = 0.f;
#pragma unroll
      for (int i = 0; i < M; ++i) sumn += ya[3 * i];
      float at[3];
      const float psum = fmaxf(wsum, cfg.gamma), dsum = wsum - psum;
      if (CONE == CONE_SOC) {
        float dl[4];
        if (adaptive) soc_contact_primal<true>(ww, wy[0], wy[1], wy[2], cfg, rp, np, dl);
        else soc_contact_primal<false>(ww, wy[0], wy[1], wy[2], cfg, rp, np, dl);
        at[0] = fmaf(cfg.mu, dl[1], dl[0]) + dsum;
        at[1] = dl[2];
        at[2] = dl[3];
      } else {
        if (adaptive) pyr_contact_primal<true>(ww, wy[0], wy[1], wy[2], cfg, rp, np);
        else pyr_contact_primal<false>(ww, wy[0], wy[1], wy[2], cfg, rp, np);
        pyr_contact_atd(ww, dsum, cfg, at);
      }
      rp = fmaxf(rp, fabsf(sumn - psum));
      float gy[6];
      g_times<NV>(Gg, ya, gy);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (adaptive) dual_component<NV, true>(Gg, 3 * ci + q, gy, wy[q], wmq[q], at[q], cfg, rho, rd, nd);
        else dual_component<NV, false>(Gg, 3 * ci + q, gy, wy[q], wmq[q], at[q], cfg, rho, rd, nd);
      }
      float rpg = 0.f, rdg = 0.f, scale[2] = {0.f, 0.f};  // group maxima (scales: adaptive rho only)
#pragma unroll
      for (int i = 0; i < M; ++i) {
        rpg = fmaxf(rpg, __shfl_sync(0xffffffffu, rp, gb + i));
        rdg = fmaxf(rdg, __shfl_sync(0xffffffffu, rd, gb + i));
      }
      if (adaptive) {
        np = fmaxf(np, fmaxf(fabsf(sumn), fabsf(psum)));
#pragma unroll
        for (int i = 0; i < M; ++i) {
          scale[0] = fmaxf(scale[0], __shfl_sync(0xffffffffu, np, gb + i));
          scale[1] = fmaxf(scale[1], __shfl_sync(0xffffffffu, nd, gb + i));
        }
      }
      const bool conv = rpg <= cfg.eps && rdg <= cfg.eps;
      const bool done = mine && (conv || it >= cfg.iters);
      if (__any_sync(0xffffffffu, done)) {
        // the finished groups' state into their records; their lane 0 writes the results
        float* rec = park + gi * L::PW;
        if (done) {
#pragma unroll
          for (int r = 0; r < 3; ++r) rec[3 * ci + r] = wy[r];
#pragma unroll
          for (int k = 0; k < WPC; ++k) rec[L::pW + WPC * ci + k] = ww[k];
          if (ci == 0) rec[L::pW + NC - 1] = wsum;
        }
        __syncwarp();
        if (done && ci == 0) {
#pragma unroll
          for (int a = 0; a < NV; ++a) y[a] = rec[a];
#pragma unroll
          for (int r = 0; r < NC; ++r) w[r] = rec[L::pW + r];
          finish(p, rpg, rdg, conv);
        }
        __syncwarp();
      }
      run = mine && !done && ci == 0;
      if (adaptive && mine && ci == 0) per(g)[L::oVote + p % S] = done ? 0.f : rho_vote(rpg, rdg, scale);
      if (done) p = -1;
    }
    if (__syncthreads_count(run) == 0) break;
    if (adaptive && __syncthreads_or(decide())) {
      // the wide lanes re-express their rows at the grasp's new rho; after the
      // rebuild they refresh their dense rows of K^-1
      const bool moved = p >= 0 && per(p / S)[L::oRho] != per(p / S)[L::oRho + 1];
      if (moved) {
        const float ratio = per(p / S)[L::oRho + 1] / per(p / S)[L::oRho];
        rescale_contact<CONE>(ww, ratio);
        wsum = rescale_sum_row(wsum, ratio, cfg.gamma);
      }
      rebuild();
      if (moved) copy_rows();
    }
  }
}

// ============================================================================ kernel: exact QPs (qp.solver = EXACT)
// One thread per QP, the minimum-norm-point solve in float32 (ExactQP); the
// block's grasps' G staged in shared memory.  Outputs: y, Q, the oracle
// calls in iters, res = (0, the final Frank-Wolfe gap, an upper bound on
// Q - Q*), z = A y clamped to the row bounds, lam = 0 (the method gives no
// multipliers); BODEX_ST_NOT_CONVERGED when the oracle-call cap stopped it.
template <int M>
__global__ void __launch_bounds__(128) qp_exact_kernel(const float* __restrict__ Gin, int B,
                                                       const float* __restrict__ T, int S, AdmmCfg cfg, float* y_out,
                                                       float* z_out, float* l_out, float* Qout, int32_t* iters_out,
                                                       int32_t* status_out, float* res_out) {
  constexpr int NV = 3 * M, NC = 9 * M + 1;
  extern __shared__ __align__(16) float smem[];
  const int GPB = blockDim.x / S;
  const size_t g0 = (size_t)blockIdx.x * GPB;
  const int ng = (int)min((size_t)GPB, (size_t)B - g0);
  for (int e = threadIdx.x; e < ng * 6 * NV; e += blockDim.x) smem[e] = Gin[g0 * 6 * NV + e];
  __syncthreads();
  const int gl = threadIdx.x / S, j = threadIdx.x % S;
  if (gl >= ng) return;
  const size_t q = (g0 + gl) * S + j;
  const float* G = smem + gl * 6 * NV;
  float t[6], y[NV], Q, gap;
#pragma unroll
  for (int r = 0; r < 6; ++r) t[r] = T[j * 6 + r];
  typename ExactQP<M>::Corral C;
  C.n = 0;
  const int ret = ExactQP<M>::solve(G, t, cfg, cfg.iters, C, y, Q, gap);
  const int calls = ret < 0 ? -ret : ret;
  bool fin = isfinite(Q);
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    y_out[q * NV + a] = y[a];
    fin = fin && isfinite(y[a]);
  }
  float sumn = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float yn = y[3 * i], yd = y[3 * i + 1], ye = y[3 * i + 2];
    sumn += yn;
    z_out[q * NC + 9 * i] = fminf(fmaxf(yn, 0.f), 1.f);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      z_out[q * NC + 9 * i + 1 + k] = fminf(fmaf(kFC[k], yd, fmaf(kFS[k], ye, -cfg.mu_c8 * yn)), 0.f);
  }
  z_out[q * NC + 9 * M] = fmaxf(sumn, cfg.gamma);
  for (int r = 0; r < NC; ++r) l_out[q * NC + r] = 0.f;
  Qout[q] = Q;
  if (iters_out) iters_out[q] = calls;
  if (res_out) {
    res_out[2 * q] = 0.f;
    res_out[2 * q + 1] = gap;
  }
  int st = 0;
  if (!fin) st |= BODEX_ST_NONFINITE;
  if (ret < 0) st |= BODEX_ST_NOT_CONVERGED;
  if (status_out) status_out[q] = st;
}

// ============================================================================ kernel: exact finish of the ADMM stragglers
// qp.polish = 2: after the ADMM kernel, the QPs it left above the residual
// target (BODEX_ST_NOT_CONVERGED) are solved exactly by the float32
// minimum-norm-point method (ExactQP).  A block takes a range of
// QP_FINISH_RANGE consecutive QPs, gathers the flagged ones into shared
// memory (ballot and prefix count), and its threads solve them one each.
// A finished QP takes the exact y and Q, gets BODEX_ST_POLISHED and loses
// BODEX_ST_NOT_CONVERGED; its z, lam, residuals and iteration count stay
// those of the ADMM run.  The QPs ADMM converged are not touched.
constexpr int QP_FINISH_RANGE = 256, QP_FINISH_THREADS = 128;

template <int M>
__global__ void __launch_bounds__(QP_FINISH_THREADS) qp_finish_kernel(const float* __restrict__ Gin, int B,
                                                                      const float* __restrict__ T, int S,
                                                                      AdmmCfg cfg, float* y_io, float* Qout,
                                                                      int32_t* status_io) {
  constexpr int NV = 3 * M;
  __shared__ int list[QP_FINISH_RANGE];
  __shared__ int count;
  const size_t n = (size_t)B * S, q0 = (size_t)blockIdx.x * QP_FINISH_RANGE;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < QP_FINISH_RANGE; k += blockDim.x) {
    const size_t q = q0 + k;
    const bool flag = q < n && (status_io[q] & BODEX_ST_NOT_CONVERGED) && !(status_io[q] & BODEX_ST_NONFINITE);
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    int base = 0;
    if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(&count, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (flag) list[base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = k;
  }
  __syncthreads();
  const int cnt = count;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const size_t q = q0 + list[i];
    const size_t b = q / S;
    const int j = (int)(q % S);
    const float* G = Gin + b * 6 * NV;
    float t[6], y[NV], Q, gap;
#pragma unroll
    for (int r = 0; r < 6; ++r) t[r] = T[j * 6 + r];
    typename ExactQP<M>::Corral C;
    C.n = 0;
    if (ExactQP<M>::solve(G, t, cfg, 64, C, y, Q, gap) < 0) continue;
#pragma unroll
    for (int a = 0; a < NV; ++a) y_io[q * NV + a] = y[a];
    Qout[q] = Q;
    status_io[q] = (status_io[q] & ~BODEX_ST_NOT_CONVERGED) | BODEX_ST_POLISHED;
  }
}

// ============================================================================ kernel: solution polishing
// A pass after qp_solve_kernel when qp.polish is set (pyramid QPs with
// eps_reg = 0): one thread per QP solves the QP exactly in FP64 by the
// minimum-norm-point method (Wolfe<M, double>), its first vertex taken at the
// ADMM point.  Where that succeeds, y and Q become the exact minimiser and
// optimum (Q to FP64 rounding, y rounded to float), the QP gets
// BODEX_ST_POLISHED and loses BODEX_ST_NOT_CONVERGED; z, lam, the residuals
// and the iteration count stay those of the ADMM run.
template <int M>
__global__ void __launch_bounds__(128) qp_polish_kernel(const float* __restrict__ Gin, int B,
                                                        const float* __restrict__ T, int S, AdmmCfg cfg, float* y_io,
                                                        float* Qout, int32_t* status_io) {
  constexpr int NV = 3 * M;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * S) return;
  if (status_io && (status_io[q] & BODEX_ST_NONFINITE)) return;
  const size_t b = q / S;
  const int j = (int)(q % S);
  const float* G = Gin + b * 6 * NV;
  float t[6], ys[NV];
  for (int r = 0; r < 6; ++r) t[r] = T[j * 6 + r];
  for (int a = 0; a < NV; ++a) ys[a] = y_io[q * NV + a];
  double yd[NV], Qd;
  if (Wolfe<M, double>::solve(G, t, cfg, ys, 1e-13, 200, yd, Qd) < 0) return;
  for (int a = 0; a < NV; ++a) y_io[q * NV + a] = (float)yd[a];
  Qout[q] = (float)Qd;
  if (status_io) status_io[q] = (status_io[q] & ~BODEX_ST_NOT_CONVERGED) | BODEX_ST_POLISHED;
}

// ============================================================================ kernel: fused evaluation / step
struct FusedArgs {
  const HandDev* hand;
  ObjDev obj;
  const float* T;
  int S, B;
  AdmmCfg cfg;
  float w_q, w_d, delta;
  float lr_t, lr_r, b1, b2, adam_eps;
  int n_steps, t0;
  // pose input (eval) or state pose (step), updated in place for step
  const float* x_in;
  float* x_state;
  float* am;
  float* av;
  float* qy;  // warm start: may be null in eval (cold start); the state's arrays in step mode
  float* qw;
  // outputs
  float* E;
  float* dEdx;
  float* Qout;
  float* yout;
  int32_t* status;
  const float* yin;  // MODE_ADJOINT: forces from a previous solve [B, s, 3m]
  float* res;        // [B] max ADMM residual of the grasp's QPs at the last step (may be null)
  int gpb;           // grasps per CTA
  int dfc;           // 1: the DFC force-closure energy |G u|^2 replaces the QPs (uniform per launch)
  int coll;          // 1: the collision energies are on (uniform per launch)
  CollDev cd;
  CollParams cp;
};

// MODE_EVAL: E and dE/dx at x.  MODE_STEP: n_steps upper iterations on the
// state.  MODE_ADJOINT: E and dE/dx at x for given forces y (no QP solve):
// the backward pass of the energy, with FK and the SDF query recomputed.
enum { MODE_EVAL = 0, MODE_STEP = 1, MODE_ADJOINT = 2 };

// The work of one CTA: GPB grasps (cta * GPB ...) of one job, s lanes each;
// threads beyond GPB * s idle but take part in every barrier.
// CONE: CONE_PYR or CONE_SOC fixes the lower-level cone at compile time;
// CONE_ANY reads it from the arguments (the several-job kernel).  ADAPT:
// whether the kernel contains the adaptive-rho solve (residual-target
// solves); kernels for fixed iteration counts leave it out, as its code
// costs the fixed loop registers.  CONE_EXACT: the pyramid's QPs solved
// exactly (qp.solver = EXACT, ExactQP) instead of by ADMM: no K^-1 set-up;
// each QP's working set (corral) carries over to the next upper step in
// the state's warm-start array: word 0 the point count, then 7 vertex
// codes, 7 fractional forces and 7 weights (component-major, like the ADMM
// iterate it replaces).
constexpr int CONE_ANY = -1;
constexpr int CONE_EXACT = 2;

template <int M, int MODE, int CONE = CONE_ANY, bool ADAPT = false>
__device__ __forceinline__ void fused_cta(const FusedArgs& A, int cta, int GPB, float* smem) {
  using L = Lay<M>;
  constexpr int NV = L::NV, NC = L::NC;
  copy_hand_to_smem(A.hand, smem);
  const int S = A.S;
  const int gl = threadIdx.x / S, lane = threadIdx.x % S;
  const int b = cta * GPB + gl;
  const bool active = (gl < GPB) && (b < A.B);
  const HandDev& H = *reinterpret_cast<const HandDev*>(smem);
  float* kin = smem + L::HAND_WORDS + gl * L::KS;
  float* per = smem + L::HAND_WORDS + GPB * L::KS + gl * L::PER;
  float* Gs = per + L::oG;
  float* xs = per + L::oX;
  float* ams = per + L::oAM;
  float* avs = per + L::oAV;
  float* sc = per + L::oSC;
  int* stat = reinterpret_cast<int*>(sc + 1);
  __syncthreads();  // hand copied
  const int D = H.D;
  const AdmmCfg& cfg = A.cfg;

  if (active) {
    const float* xsrc = (MODE == MODE_STEP) ? A.x_state : A.x_in;
    for (int k = lane; k < D; k += S) {
      xs[k] = xsrc[(size_t)b * D + k];
      if (MODE == MODE_STEP) {
        ams[k] = A.am[(size_t)b * D + k];
        avs[k] = A.av[(size_t)b * D + k];
      }
    }
    if (lane == 0) {
      *stat = 0;
      sc[2] = 0.f;      // max residual of the grasp's QPs at the last step
      sc[3] = cfg.rho;  // the grasp's ADMM penalty (adapted in solves with a residual target)
    }
  }
  // ADMM iterate of this lane's QP.  In MODE_STEP it lives in the state's
  // warm-start arrays between upper steps and in registers only around the
  // solve, so the FK / SDF / adjoint phases get the registers it would hold.
  float y[NV], w[NC];
  const size_t q = (size_t)b * S + lane, NQ = (size_t)A.B * S;
  if (MODE == MODE_ADJOINT && active) {
#pragma unroll
    for (int a = 0; a < NV; ++a) y[a] = A.yin[q * NV + a];
#pragma unroll
    for (int r = 0; r < NC; ++r) w[r] = 0.f;
  } else if (MODE == MODE_EVAL && active && A.qy && CONE != CONE_EXACT) {
#pragma unroll
    for (int a = 0; a < NV; ++a) y[a] = A.qy[a * NQ + q];
#pragma unroll
    for (int r = 0; r < NC; ++r) w[r] = A.qw[r * NQ + q];
  } else {
#pragma unroll
    for (int a = 0; a < NV; ++a) y[a] = 0.f;
#pragma unroll
    for (int r = 0; r < NC; ++r) w[r] = 0.f;
  }
  float t[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (active)
    for (int r = 0; r < 6; ++r) t[r] = A.T[lane * 6 + r];
  __syncthreads();

  const float lb1 = log2f(A.b1), lb2 = log2f(A.b2);
  for (int step = 0; step < A.n_steps; ++step) {
    // ---- A1-A3: kinematics, nearest-point query, grasp matrix (lane = contact)
    if (active && lane < M) {
      float c[3];
      fk_contact(H, lane, xs, c, per + L::oJW + lane * MAXCHAIN * 6,
                 (A.coll && A.cd.K > 0) ? per + L::oK : nullptr);  // link frames for the collision spheres
      const ContactGeo k = contact_geometry(A.obj, c);
      store_ct(per + L::oCT + L::CTW * lane, k);
      write_G_block(k, lane, NV, Gs);
      int st = 0;
      if (k.degenerate) st |= BODEX_ST_DEGENERATE_NORMAL;
      if (!finite3(k.p) || !finite3(k.n) || !isfinite(k.phi)) st |= BODEX_ST_NONFINITE;
      if (st) atomicOr(stat, st);
    }
    __syncthreads();
    // ---- constraint energies on the collision spheres (Sec. IV-B)
    if (A.coll)
      collision_phase(active, lane, S, H, A.cd, A.obj, xs, A.cp, per + L::oK, per + L::oJW, per + L::oRY,
                      per + L::oRY + 3 * A.cd.K, per + L::oRY + 3 * A.cd.K + 6 * (H.n + 1), per + L::oGC,
                      per + L::oGC + MAXD);
    // ---- A4: K^-1 per grasp (at the grasp's current penalty)
    if (MODE != MODE_ADJOINT && !A.dfc && CONE != CONE_EXACT) {
      if constexpr (ADAPT) {
        AdmmCfg cg = cfg;
        cg.rho = sc[3];
        setup_kinv<M, true>(active, lane, S, Gs, per + L::oK, kin, cg);
      } else {
        setup_kinv<M, true>(active, lane, S, Gs, per + L::oK, kin, cfg);
      }
    }
    // ---- A5: ADMM, one QP per lane
    if (active && A.dfc) per[L::oQ + lane] = 0.f;  // no lower-level QPs under DFC
    bool conv = true;
    // r_j, Q_j, the stored iterate and the status of this lane's QP
    auto finish_qp = [&]() {
      float* ry = per + L::oRY + lane * L::RYW;
      float Q = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        float s = cfg.beta * t[r];
#pragma unroll
        for (int a = 0; a < NV; ++a) s = fmaf(-Gs[r * NV + a], y[a], s);
        ry[r] = s;
        Q = fmaf(s, s, Q);
      }
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        ry[8 + a] = y[a];
        Q = fmaf(cfg.eps_reg * y[a], y[a], Q);  // regularised value when eps_reg > 0
      }
      per[L::oQ + lane] = Q;
      if (MODE == MODE_STEP && CONE != CONE_EXACT) {
#pragma unroll
        for (int a = 0; a < NV; ++a) A.qy[a * NQ + q] = y[a];
#pragma unroll
        for (int r = 0; r < NC; ++r) A.qw[r * NQ + q] = w[r];
      }
      int st = 0;
      if (cfg.eps > 0.f && !conv) st |= BODEX_ST_NOT_CONVERGED;
      if (!isfinite(Q)) st |= BODEX_ST_NONFINITE;
      if (st) atomicOr(stat, st);
    };
    const bool soc = CONE == CONE_ANY ? cfg.cone != 0 : CONE == CONE_SOC;
    if constexpr (CONE == CONE_EXACT) {
      // the exact lower level: each lane solves its QP from the corral its
      // previous step left (cold at the first step of a run)
      if (active && !A.dfc && MODE != MODE_ADJOINT) {
        typename ExactQP<M>::Corral C;
        C.n = 0;
        if (A.qw) {
          C.n = __float_as_int(A.qw[q]);
#pragma unroll
          for (int i = 0; i < ExactQP<M>::K; ++i) {
            C.V[i].code = __float_as_int(A.qw[(1 + i) * NQ + q]);
            C.V[i].frac = A.qw[(8 + i) * NQ + q];
            C.lam[i] = A.qw[(15 + i) * NQ + q];
          }
        }
        float Qx, gap;
        const int ret = ExactQP<M>::solve(Gs, t, cfg, cfg.iters, C, y, Qx, gap);
        if (A.qw) {
          A.qw[q] = __int_as_float(C.n);
#pragma unroll
          for (int i = 0; i < ExactQP<M>::K; ++i) {
            A.qw[(1 + i) * NQ + q] = __int_as_float(C.V[i].code);
            A.qw[(8 + i) * NQ + q] = C.V[i].frac;
            A.qw[(15 + i) * NQ + q] = C.lam[i];
          }
        }
        if (step == A.n_steps - 1) atomicMax(reinterpret_cast<int*>(sc + 2), __float_as_int(fmaxf(gap, 0.f)));
        if (ret < 0) atomicOr(stat, BODEX_ST_NOT_CONVERGED);
      }
      if (active && !A.dfc) finish_qp();
    } else if constexpr (ADAPT) {
      // solves with a residual target adapt rho per grasp (every thread takes
      // part); the iterate is stored with rho0 = cfg.rho and re-expressed at
      // the grasp's rho here
      if (!A.dfc) {
        float mq[NV];
        float rp = 0.f, rd = 0.f;
        AdmmCfg cg = cfg;
        cg.rho = sc[3];
        if (active) {
          if (MODE == MODE_STEP) {
#pragma unroll
            for (int a = 0; a < NV; ++a) y[a] = A.qy[a * NQ + q];
#pragma unroll
            for (int r = 0; r < NC; ++r) w[r] = A.qw[r * NQ + q];
          }
          if (MODE != MODE_ADJOINT) neg_q<M>(Gs, t, cfg.beta, mq);
          if (cg.rho != cfg.rho) {
            if (soc) rescale_w<M, CONE_SOC>(w, cfg.rho / cg.rho, cg);
            else rescale_w<M, CONE_PYR>(w, cfg.rho / cg.rho, cg);
          }
        }
        if (MODE != MODE_ADJOINT) {
          auto setup = [&](bool upd, const AdmmCfg& cc) { setup_kinv<M>(upd, lane, S, Gs, per + L::oK, kin, cc); };
          if (soc)
            admm_solve_adaptive<M, CONE_SOC>(active, lane, S, y, w, mq, kin, Gs, cg, per + L::oQ, setup, rp, rd, conv);
          else
            admm_solve_adaptive<M, CONE_PYR>(active, lane, S, y, w, mq, kin, Gs, cg, per + L::oQ, setup, rp, rd, conv);
          if (active) {
            if (lane == 0) sc[3] = cg.rho;  // every lane of the grasp holds the same rho
            if (cg.rho != cfg.rho) {
              if (soc) rescale_w<M, CONE_SOC>(w, cg.rho / cfg.rho, cg);
              else rescale_w<M, CONE_PYR>(w, cg.rho / cfg.rho, cg);
            }
            if (step == A.n_steps - 1) atomicMax(reinterpret_cast<int*>(sc + 2), __float_as_int(fmaxf(rp, rd)));
          }
        }
        if (active) finish_qp();
      }
    } else if (active && !A.dfc) {
      if (MODE == MODE_STEP) {
#pragma unroll
        for (int a = 0; a < NV; ++a) y[a] = A.qy[a * NQ + q];
#pragma unroll
        for (int r = 0; r < NC; ++r) w[r] = A.qw[r * NQ + q];
      }
      if (MODE != MODE_ADJOINT) {
        float mq[NV];
        neg_q<M>(Gs, t, cfg.beta, mq);
        float rp, rd;
        const bool last = step == A.n_steps - 1;
        if (soc) admm_solve<M, CONE_SOC>(y, w, mq, kin, Gs, cfg, rp, rd, conv, last);
        else admm_solve<M, CONE_PYR>(y, w, mq, kin, Gs, cfg, rp, rd, conv, last);
        if (step == A.n_steps - 1) atomicMax(reinterpret_cast<int*>(sc + 2), __float_as_int(fmaxf(rp, rd)));
      }
      finish_qp();
    }
    __syncthreads();
    // ---- A6: energy;  A7 (part 1), DFC only: E_Q = |G u|^2 with u = 1 on
    // every normal component, so dE/dG = 2 w_Q (G u) u^T (only the normal
    // columns), written to shared memory.  The QP energy's
    // dE/dG = -2 w_Q sum_j r_j y_j^T is formed per contact in part 2.
    if (active && A.dfc) {
      float gu[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < M; ++i) s += Gs[r * NV + 3 * i];
        gu[r] = s;
      }
      for (int e = lane; e < 6 * NV; e += S) {
        const int r = e / NV, a = e % NV;
        float g = 0.f;
#pragma unroll
        for (int rr = 0; rr < 6; ++rr) g = (rr == r) ? gu[rr] : g;
        per[L::oDG + e] = (a % 3 == 0) ? 2.f * A.w_q * g : 0.f;
      }
      if (lane == 0) {
        float EQ = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) EQ = fmaf(gu[r], gu[r], EQ);
        float Ed = 0.f;
        for (int i = 0; i < M; ++i) {
          const float r = per[L::oCT + L::CTW * i + 9] - H.alpha - A.delta;
          Ed = fmaf(r, r, Ed);
        }
        float Ec = 0.f;
        if (A.coll)
          for (int l = 0; l < S; ++l) Ec += per[L::oGC + MAXD + l];
        sc[0] = A.w_q * EQ + A.w_d * Ed + Ec;
      }
    }
    if (active && !A.dfc && lane == 0) {
      float EQ = 0.f;
      for (int j = 0; j < S; ++j) EQ += per[L::oQ + j];
      float Ed = 0.f;
      for (int i = 0; i < M; ++i) {
        const float r = per[L::oCT + L::CTW * i + 9] - H.alpha - A.delta;
        Ed = fmaf(r, r, Ed);
      }
      float Ec = 0.f;
      if (A.coll)
        for (int l = 0; l < S; ++l) Ec += per[L::oGC + MAXD + l];
      sc[0] = A.w_q * EQ + A.w_d * Ed + Ec;
    }
    // the QP energy's dE/dG is formed by the contact lanes below, from the
    // r_j and y_j the QP lanes wrote before the last barrier; only DFC's
    // shared dE/dG needs one more
    if (A.dfc) __syncthreads();
    // ---- A7 (part 2): through the contact geometry and the kinematic chain
    if (active && lane < M) {
      const ContactGeo k = load_ct(per + L::oCT + L::CTW * lane);
      float cols[18];
      if (A.dfc) {
        for (int r = 0; r < 6; ++r)
          for (int cc = 0; cc < 3; ++cc) cols[r * 3 + cc] = per[L::oDG + r * NV + 3 * lane + cc];
      } else {
        // this contact's three columns of dE/dG = -2 w_Q sum_j r_j y_j^T,
        // each entry summing j in four partial sums (j mod 4, the tail
        // into the first)
        const float* ry = per + L::oRY;
        float s[18][4];
#pragma unroll
        for (int e = 0; e < 18; ++e)
#pragma unroll
          for (int u = 0; u < 4; ++u) s[e][u] = 0.f;
        auto acc = [&](int j, int u) {
          const float4 r03 = *reinterpret_cast<const float4*>(ry + j * L::RYW);
          const float2 r45 = *reinterpret_cast<const float2*>(ry + j * L::RYW + 4);
          const float rv[6] = {r03.x, r03.y, r03.z, r03.w, r45.x, r45.y};
          const float* yj = ry + j * L::RYW + 8 + 3 * lane;
          const float yv[3] = {yj[0], yj[1], yj[2]};
#pragma unroll
          for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) s[r * 3 + cc][u] = fmaf(rv[r], yv[cc], s[r * 3 + cc][u]);
        };
        int j = 0;
        for (; j + 3 < S; j += 4) {
          acc(j, 0);
          acc(j + 1, 1);
          acc(j + 2, 2);
          acc(j + 3, 3);
        }
        for (; j < S; ++j) acc(j, 0);
#pragma unroll
        for (int e = 0; e < 18; ++e) cols[e] = -2.f * A.w_q * ((s[e][0] + s[e][1]) + (s[e][2] + s[e][3]));
      }
      float dEdc[3];
      contact_adjoint(k, cols, 2.f * A.w_d * (k.phi - H.alpha - A.delta), dEdc);
      const float* jw = per + L::oJW + lane * MAXCHAIN * 6;  // frames from the forward pass
      const float* c = k.c;
      float* cb = per + L::oCB + lane * (6 + MAXCHAIN);
      cb[0] = dEdc[0];
      cb[1] = dEdc[1];
      cb[2] = dEdc[2];
      // root rotations rx, ry, rz: axes through t
      {
        float s1, c1, s2, c2;
        angle_sincos(xs[3], &s1, &c1);
        angle_sincos(xs[4], &s2, &c2);
        const float om[3][3] = {{1.f, 0.f, 0.f}, {0.f, c1, s1}, {s2, -s1 * c2, c1 * c2}};
        const float rel[3] = {c[0] - xs[0], c[1] - xs[1], c[2] - xs[2]};
        for (int k3 = 0; k3 < 3; ++k3) {
          float v[3];
          cross3(om[k3], rel, v);
          cb[3 + k3] = dEdc[0] * v[0] + dEdc[1] * v[1] + dEdc[2] * v[2];
        }
      }
      const int Lc = H.chain_len[lane];
      for (int kk = 0; kk < Lc; ++kk) {
        const float rel[3] = {c[0] - jw[6 * kk + 3], c[1] - jw[6 * kk + 4], c[2] - jw[6 * kk + 5]};
        float v[3];
        cross3(jw + 6 * kk, rel, v);
        cb[6 + kk] = dEdc[0] * v[0] + dEdc[1] * v[1] + dEdc[2] * v[2];
      }
    }
    __syncthreads();
    // ---- gradient assembly (fixed order over contacts) and A8: Adam + clamp
    if (active) {
      const float* cb = per + L::oCB;
      const int tstep = A.t0 + step + 1;
      // bias corrections 1 - b^t as 1 - 2^(t log2 b): a function of t alone,
      // so a run split over several launches gives the same values
      const float c1 = 1.f - exp2f((float)tstep * lb1), c2 = 1.f - exp2f((float)tstep * lb2);
      const float ic1 = 1.f / c1, ic2 = 1.f / c2;  // once per step, not per coordinate
      for (int k = lane; k < D; k += S) {
        float g = 0.f;
        if (k < 6) {
          for (int i = 0; i < M; ++i) g += cb[i * (6 + MAXCHAIN) + k];
        } else {
          for (int i = 0; i < M; ++i) {
            const int pos = H.jpos[i][k - 6];
            if (pos >= 0) g += cb[i * (6 + MAXCHAIN) + 6 + pos];
          }
        }
        if (A.coll) g += per[L::oGC + k];
        if (MODE != MODE_STEP) {
          if (A.dEdx) A.dEdx[(size_t)b * D + k] = g;
        } else {
          const float mm = fmaf(A.b1, ams[k], (1.f - A.b1) * g);
          const float vv = fmaf(A.b2, avs[k], (1.f - A.b2) * g * g);
          ams[k] = mm;
          avs[k] = vv;
          const float lr = k < 3 ? A.lr_t : A.lr_r;
          const float xn = xs[k] - __fdividef(lr * (mm * ic1), sqrtf(vv * ic2) + A.adam_eps);
          xs[k] = fminf(fmaxf(xn, H.qmin[k]), H.qmax[k]);
        }
      }
    }
    __syncthreads();
  }

  // ---- write back (no early return: the several-job kernel runs this
  // function once per work item, with barriers between items)
  if (active) {
    if (lane == 0) {
      if (A.E) A.E[b] = sc[0];
      if (A.status) A.status[b] = *stat;
      if (A.res) A.res[b] = sc[2];
    }
    if (MODE == MODE_STEP) {
      for (int k = lane; k < D; k += S) {
        A.x_state[(size_t)b * D + k] = xs[k];
        A.am[(size_t)b * D + k] = ams[k];
        A.av[(size_t)b * D + k] = avs[k];
      }
    }
    if (MODE == MODE_EVAL && A.qy && CONE != CONE_EXACT) {
#pragma unroll
      for (int a = 0; a < NV; ++a) A.qy[a * NQ + q] = y[a];
#pragma unroll
      for (int r = 0; r < NC; ++r) A.qw[r * NQ + q] = w[r];
    }
    if (MODE == MODE_EVAL) {
      if (A.Qout) A.Qout[q] = per[L::oQ + lane];
      if (A.yout)
#pragma unroll
        for (int a = 0; a < NV; ++a) A.yout[q * NV + a] = y[a];
    }
  }
}

template <int M, int MODE, int CONE, bool ADAPT>
__global__ void __launch_bounds__(CTA_LANES, CONE == CONE_EXACT ? 2 : 4) fused_kernel(FusedArgs A) {
  extern __shared__ __align__(16) float smem[];
  fused_cta<M, MODE, CONE, ADAPT>(A, blockIdx.x, A.gpb, smem);
}

// ============================================================================ kernel: several jobs in one launch
// Jobs with different hand templates (m = 3, 4, 5), objects, batch sizes,
// wrench sets and step counts share one launch, every job's 200 (or n)
// upper steps inside it.  A work item is one tile of one job (the grasps of
// one CTA of that job's own launch).  Two schedules (step_params
// .work_pulling):
//   * one CTA per item, items numbered job by job in the caller's order:
//     the hardware's block scheduler hands them to SMs as slots free up;
//   * a persistent grid (PULL) of as many CTAs as fit on the GPU at once,
//     items numbered job by job in decreasing order of cost (steps x
//     wrenches x ADMM work per iteration, or steps x wrenches x contacts for
//     the exact solve): each CTA takes the next item from one global counter
//     (atomicAdd; zeroed by the host on the launch's stream before the
//     launch) until none is left.  Measured slower on the mixed-template
//     batch (the item loop costs the step registers: 488 bytes of spills at
//     the 168-register cap), so it is not the default.
// The job table travels in the kernel parameters.
struct MultiArgs {
  int n_jobs;
  int total;                            // work items
  int* counter;                         // next work item (device, zeroed before the launch)
  int m[BODEX_MAX_JOBS];
  int order_job[BODEX_MAX_JOBS];        // jobs in decreasing cost
  int order_begin[BODEX_MAX_JOBS + 1];  // first item of the k-th job in that order
  FusedArgs job[BODEX_MAX_JOBS];
};

static_assert(sizeof(MultiArgs) <= 32000, "job table must fit in the kernel parameter space");

// Work item w: the k-th job in the item order, the tile w - order_begin[k].
template <bool ADAPT, bool EXACT>
__device__ __forceinline__ void multi_item(const MultiArgs& A, int w, float* smem) {
  constexpr int CN = EXACT ? CONE_EXACT : CONE_ANY;
  int k = 0;
  while (k + 1 < A.n_jobs && w >= A.order_begin[k + 1]) ++k;
  const int j = A.order_job[k];
  const FusedArgs& J = A.job[j];
  const int cta = w - A.order_begin[k];
  switch (A.m[j]) {
    case 3: fused_cta<3, MODE_STEP, CN, ADAPT>(J, cta, J.gpb, smem); break;
    case 4: fused_cta<4, MODE_STEP, CN, ADAPT>(J, cta, J.gpb, smem); break;
    default: fused_cta<5, MODE_STEP, CN, ADAPT>(J, cta, J.gpb, smem); break;
  }
}

template <bool ADAPT, bool EXACT = false, bool PULL = false>
__global__ void __launch_bounds__(CTA_LANES, EXACT ? 2 : 4) multi_kernel(const __grid_constant__ MultiArgs A) {
  extern __shared__ __align__(16) float smem[];
  if constexpr (!PULL) {
    multi_item<ADAPT, EXACT>(A, (int)blockIdx.x, smem);  // one item per CTA, no loop
  } else {
    __shared__ int item;
#pragma unroll 1
    for (;;) {
      if (threadIdx.x == 0) item = atomicAdd(A.counter, 1);
      __syncthreads();
      const int w = item;
      __syncthreads();  // every thread has read the item before thread 0 takes the next
      if (w >= A.total) break;
      multi_item<ADAPT, EXACT>(A, w, smem);
      __syncthreads();  // shared memory is free for the next item
    }
  }
}

// ============================================================================ launch helpers
namespace bodex {

// Grasps per CTA: 96 lanes / s, capped by the shared memory one CTA may use.
template <int M>
inline int gpb_for(int s) {
  constexpr size_t kMaxSmem = 227 * 1024;
  const size_t per = 4u * (size_t)(Lay<M>::KS + Lay<M>::PER);
  const size_t fit = (kMaxSmem - 4u * Lay<M>::HAND_WORDS) / per;
  return std::max(1, std::min(CTA_LANES / s, (int)fit));
}

// Grasps per CTA of the batched QP kernel: 96 lanes / s, capped by its
// shared memory.
template <int M, int CONE>
inline int qp_gpb(int s) {
  constexpr size_t kMaxSmem = 227 * 1024;
  using L = LayQP<M, CONE>;
  const size_t per = 4u * (size_t)(L::KS + L::PER + s * L::PW);
  return std::max(1, std::min(CTA_LANES / s, (int)((kMaxSmem - 128) / per)));
}

// Grasps per CTA: the requested count (autotuner), else the default,
// never more than fit in 96 lanes and in shared memory.
template <int M>
inline int pick_gpb(int s, int requested) {
  const int cap = gpb_for<M>(s);
  return requested > 0 ? std::min(requested, cap) : cap;
}

// Raises the kernel's dynamic shared-memory limit when needed, once per
// device and size (so that launches recorded into a CUDA graph issue no
// attribute calls after the first).
template <class K>
inline int ensure_smem(K kernel, size_t bytes) {
  // A launch reports errors through cudaGetLastError; clear what an earlier,
  // already reported failure may have left behind (sticky device faults are
  // returned again by the next call regardless).
  (void)cudaGetLastError();
  if (bytes <= 48 * 1024) return BODEX_OK;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> configured;  // (kernel, device) -> bytes
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = configured.find(key);
  if (it != configured.end() && it->second >= bytes) return BODEX_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_fail(e, "cudaFuncSetAttribute");
  }
  configured[key] = bytes;
  return BODEX_OK;
}

}  // namespace bodex

template <int M>
inline int run_fused(int mode, const FusedArgs& A0, cudaStream_t st) {
  FusedArgs A = A0;
  A.gpb = pick_gpb<M>(A.S, A0.gpb);
  const int gpb = A.gpb;
  const size_t bytes = Lay<M>::bytes(gpb);
  const dim3 grid((A.B + gpb - 1) / gpb), block(gpb * A.S);
  if (A.B == 0) return BODEX_OK;
  const bool soc = A.cfg.cone != 0;
  const bool adapt = A.cfg.eps > 0.f && A.cfg.adapt;
  auto go = [&](auto kernel) -> int {
    if (int r = ensure_smem(kernel, bytes)) return r;
    kernel<<<grid, block, bytes, st>>>(A);
    return BODEX_OK;
  };
  int r;
  if (mode == MODE_ADJOINT) r = go(fused_kernel<M, MODE_ADJOINT, CONE_PYR, false>);  // no lower-level solve
  else if (A.cfg.solver == BODEX_QP_EXACT)
    r = mode == MODE_STEP ? go(fused_kernel<M, MODE_STEP, CONE_EXACT, false>) : go(fused_kernel<M, MODE_EVAL, CONE_EXACT, false>);
  else if (mode == MODE_STEP)
    r = soc ? (adapt ? go(fused_kernel<M, MODE_STEP, CONE_SOC, true>) : go(fused_kernel<M, MODE_STEP, CONE_SOC, false>))
            : (adapt ? go(fused_kernel<M, MODE_STEP, CONE_PYR, true>) : go(fused_kernel<M, MODE_STEP, CONE_PYR, false>));
  else
    r = soc ? (adapt ? go(fused_kernel<M, MODE_EVAL, CONE_SOC, true>) : go(fused_kernel<M, MODE_EVAL, CONE_SOC, false>))
            : (adapt ? go(fused_kernel<M, MODE_EVAL, CONE_PYR, true>) : go(fused_kernel<M, MODE_EVAL, CONE_PYR, false>));
  if (r) return r;
  return launch_err("fused_kernel launch");
}

template <int M>
inline int run_qp(const float* G, int B, const float* T, int s, const AdmmCfg& cfg, int warm, float* y, float* z,
           float* lam, float* Q, int32_t* iters, int32_t* status, float* res, cudaStream_t st) {
  if (B == 0) return BODEX_OK;
  if (cfg.solver == BODEX_QP_EXACT) {
    const int gpb = std::max(1, 128 / s);
    const size_t bytes = 4u * (size_t)gpb * 6 * 3 * M;
    qp_exact_kernel<M><<<(B + gpb - 1) / gpb, gpb * s, bytes, st>>>(G, B, T, s, cfg, y, z, lam, Q, iters, status,
                                                                    res);
    return launch_err("qp_exact_kernel launch");
  }
  const int gpb = cfg.cone ? qp_gpb<M, CONE_SOC>(s) : qp_gpb<M, CONE_PYR>(s);
  const size_t bytes = cfg.cone ? LayQP<M, CONE_SOC>::bytes(gpb, s) : LayQP<M, CONE_PYR>::bytes(gpb, s);
  if (cfg.cone) {
    if (int r = ensure_smem(qp_solve_kernel<M, CONE_SOC>, bytes)) return r;
    qp_solve_kernel<M, CONE_SOC><<<(B + gpb - 1) / gpb, gpb * s, bytes, st>>>(G, B, T, s, cfg, warm, y, z, lam, Q,
                                                                              iters, status, res);
  } else {
    if (int r = ensure_smem(qp_solve_kernel<M, CONE_PYR>, bytes)) return r;
    qp_solve_kernel<M, CONE_PYR><<<(B + gpb - 1) / gpb, gpb * s, bytes, st>>>(G, B, T, s, cfg, warm, y, z, lam, Q,
                                                                              iters, status, res);
    if (int r = launch_err("qp_solve_kernel launch")) return r;
    if (cfg.polish == 1 && cfg.eps_reg == 0.f) {
      const size_t n = (size_t)B * s;
      qp_polish_kernel<M><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(G, B, T, s, cfg, y, Q, status);
      return launch_err("qp_polish_kernel launch");
    }
    if (cfg.polish == 2 && cfg.eps_reg == 0.f && cfg.eps > 0.f && status) {
      const size_t n = (size_t)B * s;
      qp_finish_kernel<M><<<(unsigned)((n + QP_FINISH_RANGE - 1) / QP_FINISH_RANGE), QP_FINISH_THREADS, 0, st>>>(
          G, B, T, s, cfg, y, Q, status);
      return launch_err("qp_finish_kernel launch");
    }
    return BODEX_OK;
  }
  return launch_err("qp_solve_kernel launch");
}

// Launchers, one translation unit each (fused_m*.cu, qp.cu, fused_multi.cu).
int launch_fused_m3(int mode, const FusedArgs& A, cudaStream_t st);
int launch_fused_m4(int mode, const FusedArgs& A, cudaStream_t st);
int launch_fused_m5(int mode, const FusedArgs& A, cudaStream_t st);
int launch_qp(int m, const float* G, int B, const float* T, int s, const AdmmCfg& cfg, int warm, float* y, float* z,
              float* lam, float* Q, int32_t* iters, int32_t* status, float* res, cudaStream_t st);
int launch_multi(bool adapt, bool exact, bool pull, const MultiArgs& MA, size_t bytes, cudaStream_t st);
