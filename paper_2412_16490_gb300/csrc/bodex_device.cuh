// Device-side building blocks of the BODex coarse-stage hot path (sm_103a).
//
// Everything here is float32 CUDA-core arithmetic.  The lower-level QPs are
// tiny dense problems with a different matrix per grasp, so the path is not a
// shared dense contraction and does not use the tensor cores; the per-grasp
// data (G, K^-1) lives in shared memory and the per-QP ADMM iterate in
// registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bodex.h"

namespace bodex {

constexpr int MAXJ = BODEX_MAX_JOINTS;
constexpr int MAXM = BODEX_MAX_CONTACTS;
constexpr int MAXCHAIN = BODEX_MAX_CHAIN;
constexpr int MAXD = 6 + MAXJ;
constexpr int SMAX = 16;  // wrenches per grasp

// cos / sin of pi/8: the facet normals of the 8-edge pyramid sit at
// phi_k = (2k+1) pi/8 in the contact's (d, e) plane.
constexpr float C8 = 0.92387953251128674f;
constexpr float S8 = 0.38268343236508978f;

// ------------------------------------------------------------------ handles
struct HandDev {
  int n, m, D, S;
  float alpha;
  int parent[MAXJ];
  alignas(16) float offset[MAXJ][12];  // rows [R_r0 R_r1 R_r2 t_r], one float4 each
  float axis[MAXJ][3];
  float qmin[MAXD], qmax[MAXD];
  int clink[MAXM];
  float clocal[MAXM][3];
  int chain_len[MAXM];
  int chain[MAXM][MAXCHAIN];  // joints from the root to contact i's link
  int8_t jpos[MAXM][MAXJ];    // position of joint j in contact i's chain, or -1
};

// Collision spheres of a hand (device arrays, read through the read-only
// cache).  Spheres are ordered by slot: slot L < n is link L, slot n the
// root; slot L holds spheres slot_start[L] .. slot_start[L+1]-1 and has a
// bounding sphere sbound[L] (in its frame) around them.  The slots whose
// spheres pair with slot L's for self-penetration are
// spartners[spstart[L] .. spstart[L+1]-1] (each slot pair appears under both).
struct CollDev {
  int K;
  const float4* sph;     // [K] centre in the link frame (xyz), radius (w)
  const float4* sbound;  // [n+1] bounding sphere of the slot's spheres
  const int* slot_start;
  const int* spstart;
  const int* spartners;
};

struct CollParams {
  float w_pen, w_self, w_lim, eta_pen, eta_lim;
};

struct ObjDev {
  int kind;  // 0 sphere, 1 grid
  float cx, cy, cz, r;
  int N;
  float h, inv_h;
  float ox, oy, oz;
  const float* grid;
  float gcx, gcy, gcz;  // gravity centre
};

struct AdmmCfg {
  float mu_c8;  // mu cos(pi/8)
  float mu;
  int cone;     // 0: the 8-facet pyramid, 1: the elliptic cone
  int adapt;    // adapt rho per grasp in solves with a residual target
  float beta, gamma, rho, sigma, alpha, eps, eps_reg;
  int iters, check;
  int fp64_setup;  // build K^-1 in double (set by the host per launch)
  int polish;      // polish converged pyramid QPs (bodex_qp_solve_batch)
  int solver;      // BODEX_QP_ADMM or BODEX_QP_EXACT
};

__host__ __device__ inline AdmmCfg admm_cfg(const bodex_qp_params& p) {
  AdmmCfg c;
  c.mu_c8 = p.mu * C8;
  c.mu = p.mu;
  c.cone = p.cone;
  c.adapt = p.adaptive_rho;
  c.beta = p.beta;
  c.gamma = p.gamma;
  c.rho = p.rho;
  c.sigma = p.sigma;
  c.alpha = p.alpha;
  c.eps = p.eps_abs;
  c.eps_reg = p.eps_reg;
  c.iters = p.max_iter;
  c.check = p.check_every > 0 ? p.check_every : 10;
  c.fp64_setup = 0;
  c.polish = p.polish;
  c.solver = p.solver;
  return c;
}

// ------------------------------------------------------------------ rigid transforms
struct Tf {
  float R[9];
  float t[3];
};

__device__ __forceinline__ void tf_mul(const Tf& A, const Tf& B, Tf& C) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C.R[3 * r + c] = fmaf(A.R[3 * r], B.R[c], fmaf(A.R[3 * r + 1], B.R[3 + c], A.R[3 * r + 2] * B.R[6 + c]));
    C.t[r] = fmaf(A.R[3 * r], B.t[0], fmaf(A.R[3 * r + 1], B.t[1], fmaf(A.R[3 * r + 2], B.t[2], A.t[r])));
  }
}

__device__ __forceinline__ void rot_vec(const float* R, const float* v, float* o) {
  o[0] = fmaf(R[0], v[0], fmaf(R[1], v[1], R[2] * v[2]));
  o[1] = fmaf(R[3], v[0], fmaf(R[4], v[1], R[5] * v[2]));
  o[2] = fmaf(R[6], v[0], fmaf(R[7], v[1], R[8] * v[2]));
}

// sin and cos of a joint or root angle: x is reduced to [-pi, pi] by
// x - 2 pi k, k = rint(x / 2 pi), with 2 pi split into its float value and
// the remainder (-1.748e-7), and the hardware approximation evaluates sin
// and cos there (absolute error about 4e-7 on [-pi, pi]).  The clamp of
// Eq. (4) keeps the angles within a few radians, where the reduction is
// accurate to float rounding.
__device__ __forceinline__ void angle_sincos(float x, float* s, float* c) {
  const float k = rintf(x * 0.159154943091895336f);
  float r = fmaf(-k, 6.28318548202514648f, x);
  r = fmaf(-k, -1.74845560007444870e-7f, r);
  __sincosf(r, s, c);
}

// Rotation by q about the unit axis a (Rodrigues).
__device__ __forceinline__ void rodrigues(const float* a, float q, float* R) {
  float s, c;
  angle_sincos(q, &s, &c);
  const float C = 1.0f - c;
  R[0] = c + a[0] * a[0] * C;
  R[1] = a[0] * a[1] * C - a[2] * s;
  R[2] = a[0] * a[2] * C + a[1] * s;
  R[3] = a[1] * a[0] * C + a[2] * s;
  R[4] = c + a[1] * a[1] * C;
  R[5] = a[1] * a[2] * C - a[0] * s;
  R[6] = a[2] * a[0] * C - a[1] * s;
  R[7] = a[2] * a[1] * C + a[0] * s;
  R[8] = c + a[2] * a[2] * C;
}

// Root frame Trans(t) Rx(rx) Ry(ry) Rz(rz) and the world axes of the three
// virtual revolute joints (rx about world X, ry about Rx Y, rz about Rx Ry Z).
__device__ __forceinline__ void root_frame(const float* x, Tf& T, float om[3][3]) {
  float s1, c1, s2, c2, s3, c3;
  angle_sincos(x[3], &s1, &c1);
  angle_sincos(x[4], &s2, &c2);
  angle_sincos(x[5], &s3, &c3);
  T.R[0] = c2 * c3;
  T.R[1] = -c2 * s3;
  T.R[2] = s2;
  T.R[3] = s1 * s2 * c3 + c1 * s3;
  T.R[4] = -s1 * s2 * s3 + c1 * c3;
  T.R[5] = -s1 * c2;
  T.R[6] = -c1 * s2 * c3 + s1 * s3;
  T.R[7] = c1 * s2 * s3 + s1 * c3;
  T.R[8] = c1 * c2;
  T.t[0] = x[0];
  T.t[1] = x[1];
  T.t[2] = x[2];
  om[0][0] = 1.f; om[0][1] = 0.f; om[0][2] = 0.f;
  om[1][0] = 0.f; om[1][1] = c1;  om[1][2] = s1;
  om[2][0] = s2;  om[2][1] = -s1 * c2; om[2][2] = c1 * c2;
}

__device__ __forceinline__ void store_frame(const Tf& T, float* f) {
#pragma unroll
  for (int e = 0; e < 9; ++e) f[e] = T.R[e];
  f[9] = T.t[0];
  f[10] = T.t[1];
  f[11] = T.t[2];
}

// Forward kinematics of contact i's link (Sec. IV-B): walks the chain from
// the root and returns the link frame T; if `jw` is given, stores the world
// axis and a point on the axis of every chain joint (6 floats each, in chain
// order) for the adjoint.
__device__ inline void fk_link(const HandDev& H, int i, const float* x, Tf& T, float* jw, float* frames = nullptr) {
  float om[3][3];
  root_frame(x, T, om);
  if (frames) store_frame(T, frames + 12 * H.n);  // the root
  const int L = H.chain_len[i];
  for (int k = 0; k < L; ++k) {
    const int j = H.chain[i][k];
    Tf off;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float4 o = reinterpret_cast<const float4*>(H.offset[j])[r];
      off.R[3 * r] = o.x, off.R[3 * r + 1] = o.y, off.R[3 * r + 2] = o.z;
      off.t[r] = o.w;
    }
    Tf base;
    tf_mul(T, off, base);
    const float a[3] = {H.axis[j][0], H.axis[j][1], H.axis[j][2]};
    if (jw) {
      rot_vec(base.R, a, jw + 6 * k);
      jw[6 * k + 3] = base.t[0];
      jw[6 * k + 4] = base.t[1];
      jw[6 * k + 5] = base.t[2];
    }
    Tf rq;
    rodrigues(a, x[6 + j], rq.R);
    rq.t[0] = rq.t[1] = rq.t[2] = 0.f;
    tf_mul(base, rq, T);
    if (frames) store_frame(T, frames + 12 * j);
  }
}

__device__ __forceinline__ void tf_point(const Tf& T, const float* p, float* c) {
  c[0] = fmaf(T.R[0], p[0], fmaf(T.R[1], p[1], fmaf(T.R[2], p[2], T.t[0])));
  c[1] = fmaf(T.R[3], p[0], fmaf(T.R[4], p[1], fmaf(T.R[5], p[2], T.t[1])));
  c[2] = fmaf(T.R[6], p[0], fmaf(T.R[7], p[1], fmaf(T.R[8], p[2], T.t[2])));
}

// Contact point c_{i,w} = R c_{i,l} + T of contact i (and chain frames, see
// fk_link; `frames`, if given, receives the frame of every chain link at
// 12 j and the root frame at 12 n, row-major [R | t]).
__device__ inline void fk_contact(const HandDev& H, int i, const float* x, float* c, float* jw,
                                  float* frames = nullptr) {
  Tf T;
  fk_link(H, i, x, T, jw, frames);
  const float* cl = H.clocal[i];
  c[0] = fmaf(T.R[0], cl[0], fmaf(T.R[1], cl[1], fmaf(T.R[2], cl[2], T.t[0])));
  c[1] = fmaf(T.R[3], cl[0], fmaf(T.R[4], cl[1], fmaf(T.R[5], cl[2], T.t[1])));
  c[2] = fmaf(T.R[6], cl[0], fmaf(T.R[7], cl[1], fmaf(T.R[8], cl[2], T.t[2])));
}

// ------------------------------------------------------------------ SDF query
// phi, gradient g, Hessian h (xx, xy, xz, yy, yz, zz) and voxel cell at c.
// Grid: node-sampled trilinear interpolant; outside the node box
// phi(c) = phi(clamp(c)) + |c - clamp(c)| with the exact derivatives of that
// expression.
struct SdfQ {
  float phi;
  float g[3];
  float h[6];
  int cell[3];
};

__device__ inline SdfQ sdf_query(const ObjDev& O, const float* c) {
  SdfQ q;
  if (O.kind == 0) {
    const float v0 = c[0] - O.cx, v1 = c[1] - O.cy, v2 = c[2] - O.cz;
    const float L = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    const float iL = 1.0f / L;
    const float u0 = v0 * iL, u1 = v1 * iL, u2 = v2 * iL;
    q.phi = L - O.r;
    q.g[0] = u0; q.g[1] = u1; q.g[2] = u2;
    q.h[0] = (1.f - u0 * u0) * iL;
    q.h[1] = -u0 * u1 * iL;
    q.h[2] = -u0 * u2 * iL;
    q.h[3] = (1.f - u1 * u1) * iL;
    q.h[4] = -u1 * u2 * iL;
    q.h[5] = (1.f - u2 * u2) * iL;
    q.cell[0] = q.cell[1] = q.cell[2] = 0;
    return q;
  }
  const int N = O.N;
  const float org[3] = {O.ox, O.oy, O.oz};
  const float hi_off = O.h * (float)(N - 1);
  float cl[3], t[3], dv[3];
  bool cla[3];
  int cell[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = org[a], hi = org[a] + hi_off;
    cla[a] = (c[a] < lo) || (c[a] > hi);
    cl[a] = fminf(fmaxf(c[a], lo), hi);
    const float u = (cl[a] - org[a]) / O.h;
    int k = (int)floorf(u);
    k = min(max(k, 0), N - 2);
    cell[a] = k;
    t[a] = u - (float)k;
    dv[a] = c[a] - cl[a];
  }
  const float* G0 = O.grid + ((size_t)cell[2] * N + cell[1]) * N + cell[0];
  const size_t sy = N, sz = (size_t)N * N;
  const float v000 = __ldg(G0), v100 = __ldg(G0 + 1);
  const float v010 = __ldg(G0 + sy), v110 = __ldg(G0 + sy + 1);
  const float v001 = __ldg(G0 + sz), v101 = __ldg(G0 + sz + 1);
  const float v011 = __ldg(G0 + sz + sy), v111 = __ldg(G0 + sz + sy + 1);
  const float tx = t[0], ty = t[1], tz = t[2];
  // interpolate along x, then y, then z
  const float a00 = fmaf(tx, v100 - v000, v000), a10 = fmaf(tx, v110 - v010, v010);
  const float a01 = fmaf(tx, v101 - v001, v001), a11 = fmaf(tx, v111 - v011, v011);
  const float b0 = fmaf(ty, a10 - a00, a00), b1 = fmaf(ty, a11 - a01, a01);
  const float phi_cl = fmaf(tz, b1 - b0, b0);
  // d/dx: differences along x, interpolated in y, z
  const float dx00 = v100 - v000, dx10 = v110 - v010, dx01 = v101 - v001, dx11 = v111 - v011;
  const float dxb0 = fmaf(ty, dx10 - dx00, dx00), dxb1 = fmaf(ty, dx11 - dx01, dx01);
  const float gx = fmaf(tz, dxb1 - dxb0, dxb0) * O.inv_h;
  const float gy = fmaf(tz, a11 - a01 - (a10 - a00), a10 - a00) * O.inv_h;
  const float gz = (b1 - b0) * O.inv_h;
  // mixed second derivatives (the pure ones vanish for a trilinear cell)
  const float hxy = fmaf(tz, (dx11 - dx01) - (dx10 - dx00), dx10 - dx00) * O.inv_h * O.inv_h;
  const float hxz = (dxb1 - dxb0) * O.inv_h * O.inv_h;
  const float hyz = ((a11 - a01) - (a10 - a00)) * O.inv_h * O.inv_h;
  const float gcl[3] = {gx, gy, gz};
  const float hcl[6] = {0.f, hxy, hxz, 0.f, hyz, 0.f};
  const float dl2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
  const bool any = cla[0] || cla[1] || cla[2];
  const float dl = any ? sqrtf(dl2) : 0.f;
  const float idl = any ? 1.0f / dl : 0.f;
  q.phi = phi_cl + dl;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    q.g[a] = cla[a] ? dv[a] * idl : gcl[a];
    q.cell[a] = cell[a];
  }
  // Hessian entries (a, b) in order xx, xy, xz, yy, yz, zz
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int a = ia[e], b = ib[e];
    float v = 0.f;
    if (!cla[a] && !cla[b]) v = hcl[e];
    else if (cla[a] && cla[b]) v = ((a == b ? 1.f : 0.f) - dv[a] * dv[b] * idl * idl) * idl;
    q.h[e] = v;
  }
  return q;
}

// Tangent basis (d, e) of a unit normal n with n = d x e: the branch-free
// construction of Duff et al., "Building an Orthonormal Basis, Revisited"
// (JCGT 2017), sign taken from n_z.
__device__ __forceinline__ void tangent_basis(const float* n, float* d, float* e) {
  const float sg = copysignf(1.0f, n[2]);
  const float a = __fdividef(-1.0f, sg + n[2]);  // |sg + n_z| >= 1
  const float b = n[0] * n[1] * a;
  d[0] = 1.0f + sg * n[0] * n[0] * a;
  d[1] = sg * b;
  d[2] = -sg * n[0];
  e[0] = b;
  e[1] = sg + n[1] * n[1] * a;
  e[2] = -n[1];
}

__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Per-contact geometry kept between the forward pass and the adjoint.
struct ContactGeo {
  float c[3], p[3], n[3];  // p relative to the gravity centre
  float phi, g[3], h[6];
  int cell[3];
  int degenerate;
};

// Nearest-point query (Sec. IV-B): p = c - phi g/|g|, inward n = -g/|g|.
__device__ inline ContactGeo contact_geometry(const ObjDev& O, const float* c) {
  ContactGeo k;
  const SdfQ q = sdf_query(O, c);
  const float L2 = q.g[0] * q.g[0] + q.g[1] * q.g[1] + q.g[2] * q.g[2];
  k.degenerate = !(L2 >= 1e-24f);
  const float iL = rsqrtf(L2);
  const float gc[3] = {O.gcx, O.gcy, O.gcz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float no = q.g[a] * iL;
    k.c[a] = c[a];
    k.n[a] = -no;
    k.p[a] = (c[a] - q.phi * no) - gc[a];
    k.g[a] = q.g[a];
    k.cell[a] = q.cell[a];
  }
  k.phi = q.phi;
#pragma unroll
  for (int e = 0; e < 6; ++e) k.h[e] = q.h[e];
  return k;
}

// Columns 3i..3i+2 of the grasp matrix (Sec. III, Eq. (2)):
// [n d e ; p x n, p x d, p x e], written to G (6 x nv, row-major).
__device__ __forceinline__ void write_G_block(const ContactGeo& k, int i, int nv, float* G) {
  float d[3], e[3];
  tangent_basis(k.n, d, e);
  const float* cols[3] = {k.n, d, e};
#pragma unroll
  for (int cidx = 0; cidx < 3; ++cidx) {
    float tq[3];
    cross3(k.p, cols[cidx], tq);
    const int col = 3 * i + cidx;
    G[0 * nv + col] = cols[cidx][0];
    G[1 * nv + col] = cols[cidx][1];
    G[2 * nv + col] = cols[cidx][2];
    G[3 * nv + col] = tq[0];
    G[4 * nv + col] = tq[1];
    G[5 * nv + col] = tq[2];
  }
}

// Sizes of one QP with M contacts.
template <int M>
struct Admm {
  static constexpr int NV = 3 * M;
  static constexpr int NC = 9 * M + 1;
  static constexpr int NVP = (NV + 3) & ~3;
  // K^-1 is symmetric: only its upper triangle is stored, row-major and
  // packed (entry (a, b), a <= b, at tri(a, b)), padded to whole float4s
  static constexpr int NTRI = NV * (NV + 1) / 2;
  static constexpr int NTRI4 = (NTRI + 3) / 4;
  static constexpr __host__ __device__ int tri(int a, int b) { return a * NV - (a * (a - 1)) / 2 + (b - a); }
};

// ------------------------------------------------------------------ QP setup
// K = P + sigma I + rho A^T A with P = 2 G^T G (+ 2 eps_reg I).  For the
// pyramid rows A^T A is the constant
//   diag per contact (1 + 8 mu^2 cos^2(pi/8), 4, 4)  (f_n row + 8 facets)
//   + u u^T, u = indicator of the normal components   (the sum row),
// because the facet normals sum to zero and their squares sum to 4 per
// axis.  Hence K = Dg + V V^T with Dg diagonal and V = [sqrt2 G^T, sqrt(rho) u]
// of rank 7, and by the Sherman-Morrison-Woodbury identity
//   K^-1 = Dg^-1 - U U^T,   U = Dg^-1 V L^-T,   L L^T = I + V^T Dg^-1 V (7 x 7).
// Every lane of the grasp takes part; no lane factors the 3m x 3m matrix.
struct DiagK {
  float dn, dt;  // Dg for a normal / a tangential component
};
__device__ __forceinline__ DiagK diag_k(const AdmmCfg& c) {
  DiagK d;
  const float base = fmaf(2.f, c.eps_reg, c.sigma);
  if (c.cone) {  // rows f_n and (mu f_n, f_d, f_e): A^T A = diag(1 + mu^2, 1, 1)
    d.dn = fmaf(c.rho, fmaf(c.mu, c.mu, 1.f), base);
    d.dt = base + c.rho;
  } else {
    d.dn = fmaf(c.rho, fmaf(8.f * c.mu_c8, c.mu_c8, 1.f), base);
    d.dt = fmaf(4.f, c.rho, base);
  }
  return d;
}

// Fused multiply-add in float or double.  The QP setup, the ADMM iteration
// and its residuals spell every multiply-add out (fmaf / fma_r) and leave no
// `a * b + c` to the compiler's contraction, whose choice can depend on the
// code a function is inlined into: kernels that inline the same solve in
// different contexts then give bitwise equal results.
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }

// Entry e (0..27, row-major upper triangle of the 7x7) of M = I + V^T Dg^-1 V,
// accumulated in precision R; idn / idt are 1 / Dg of a normal / a
// tangential component.
template <int M, typename R>
__device__ inline R woodbury_M_entry(const float* G, int e, const AdmmCfg& c, R idn, R idt) {
  constexpr int NV = 3 * M;
  // rows of the 7 x 7 upper triangle start at entries 0, 7, 13, 18, 22, 25, 27
  const int a = (e >= 7) + (e >= 13) + (e >= 18) + (e >= 22) + (e >= 25) + (e >= 27);
  const int b = e - (a * 7 - (a * (a - 1)) / 2) + a;
  if (b < 6) {  // both columns from sqrt2 G^T: normal and tangential parts summed apart
    R sn = 0, st = 0;
#pragma unroll
    for (int i = 0; i < NV; i += 3) {
      sn = fma_r(R(G[a * NV + i]), R(G[b * NV + i]), sn);
      st = fma_r(R(G[a * NV + i + 1]), R(G[b * NV + i + 1]), st);
      st = fma_r(R(G[a * NV + i + 2]), R(G[b * NV + i + 2]), st);
    }
    return fma_r(R(2), fma_r(sn, idn, st * idt), a == b ? R(1) : R(0));
  }
  R s = 0;
  if (a < 6) {  // sqrt2 G^T against sqrt(rho) u
#pragma unroll
    for (int i = 0; i < NV; i += 3) s += R(G[a * NV + i]);
    return s * (sqrt(R(2) * R(c.rho)) * idn);
  }
  return fma_r(R(c.rho) * R(M), idn, R(1));
}

// Scratch (in floats) that setup_kinv_woodbury<M, R> needs: M (28), then U
// in rows of 8 (16-byte aligned when the scratch is).
template <int M, typename R>
struct WoodburyScratch {
  static constexpr int floats = (28 + 8 * 3 * M) * (int)(sizeof(R) / 4);
};

// Row i of U (7 entries, stored in a row of 8) in registers.
template <typename R>
__device__ __forceinline__ void load_u_row(const R* Us, int i, R (&u)[7]) {
  if constexpr (sizeof(R) == 4) {
    const float4 lo = *reinterpret_cast<const float4*>(Us + 8 * i);
    const float4 hi = *reinterpret_cast<const float4*>(Us + 8 * i + 4);
    u[0] = lo.x, u[1] = lo.y, u[2] = lo.z, u[3] = lo.w, u[4] = hi.x, u[5] = hi.y, u[6] = hi.z;
  } else {
#pragma unroll
    for (int a = 0; a < 7; a += 2) {
      const double2 v = *reinterpret_cast<const double2*>(Us + 8 * i + a);
      u[a] = v.x;
      if (a + 1 < 7) u[a + 1] = v.y;
    }
  }
}

// Writes alpha K^-1 (alpha: the ADMM relaxation; packed upper triangle, see
// Admm<M>::tri; rounded to float) for one grasp,
// computed in precision R: float for the fixed-iteration step loop, double
// when the solve iterates to a residual target (the ADMM fixed point moves
// with the backward error of the inverse: the dual residual floor is
// |(K^-1_computed)^-1 - K| |y|).  The scratch must be 16-byte aligned.
// Must be called by every thread of the CTA (contains barriers).
// UNROLL: for 12 lanes per grasp in float, the M entries and the rows of U
// are formed in unrolled rounds (the fused step, which repeats the set-up
// every upper step; the QP kernels set up once and keep the loops, which
// need fewer registers next to their repacking state).
template <int M, typename R, bool UNROLL = false>
__device__ inline void setup_kinv_woodbury(bool active, int lane, int S, const float* G, float* scratch, float* Kinv,
                                           const AdmmCfg& c) {
  constexpr int NV = 3 * M;
  const DiagK dk = diag_k(c);
  R* Ms = reinterpret_cast<R*>(scratch);  // 28
  R* Us = Ms + 28;                        // NV rows of 8
  const R idn = R(1) / R(dk.dn), idt = R(1) / R(dk.dt);
  if (active) {
    if (UNROLL && sizeof(R) == 4 && S == 12) {
      // 12 lanes (the paper's wrench set): three rounds, every value formed
      // before any store so that the rounds' loads overlap (measured 1.8%
      // faster per fused step together with the same form of the U rows)
      R v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = lane + 12 * k < 28 ? woodbury_M_entry<M, R>(G, lane + 12 * k, c, idn, idt) : R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (lane + 12 * k < 28) Ms[lane + 12 * k] = v[k];
    } else {
      for (int e = lane; e < 28; e += S) Ms[e] = woodbury_M_entry<M, R>(G, e, c, idn, idt);
    }
  }
  __syncthreads();
  // 7x7 Cholesky.  Index (a, b), a <= b, of the row-major upper triangle;
  // after factoring, entry (a, b) holds L[b][a].  In float every lane
  // factors its own copy in registers (no barrier); in double, whose
  // arithmetic is far slower, lane 0 factors it once into the shared M and
  // ild (in Us' padding column) and the lanes read it back.
  auto idx = [](int a, int b) { return a * 7 - (a * (a - 1)) / 2 + (b - a); };
  R L[28];
  R ild[7];  // reciprocals of the diagonal of L
  auto factor = [&]() {
    if constexpr (sizeof(R) == 4) {  // seven 16-byte loads (the scratch is 16-byte aligned)
#pragma unroll
      for (int e = 0; e < 28; e += 4) {
        const float4 v = *reinterpret_cast<const float4*>(Ms + e);
        L[e] = v.x, L[e + 1] = v.y, L[e + 2] = v.z, L[e + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 28; ++e) L[e] = Ms[e];
    }
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      R d = L[idx(j, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) d = fma_r(-L[idx(k, j)], L[idx(k, j)], d);
      const R dd = d > R(1e-30) ? d : R(1e-30);
      R il;
      if constexpr (sizeof(R) == 4) {  // one reciprocal square root; only 1 / l_jj is used below
        il = rsqrtf(dd);
        L[idx(j, j)] = dd * il;
      } else {
        const R ljj = sqrt(dd);
        L[idx(j, j)] = ljj;
        il = R(1) / ljj;
      }
      ild[j] = il;
#pragma unroll
      for (int i = j + 1; i < 7; ++i) {
        R t = L[idx(j, i)];
#pragma unroll
        for (int k = 0; k < j; ++k) t = fma_r(-L[idx(k, i)], L[idx(k, j)], t);
        L[idx(j, i)] = t * il;
      }
    }
  };
  if constexpr (sizeof(R) == 8) {
    if (active && lane == 0) {
      factor();
#pragma unroll
      for (int e = 0; e < 28; ++e) Ms[e] = L[e];
#pragma unroll
      for (int a = 0; a < 7; ++a) Us[a * 8 + 7] = ild[a];
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int e = 0; e < 28; ++e) L[e] = Ms[e];
#pragma unroll
      for (int a = 0; a < 7; ++a) ild[a] = Us[a * 8 + 7];  // the U rows below write entries 0..6 only
    }
  } else {
    if (active) factor();
  }
  if (active) {
    const R s2 = sqrt(R(2)), sr = sqrt(R(c.rho));
    // row i of U: w = Dg^-1 V_i (V_i = [sqrt2 G^T, sqrt(rho) u] row i), then
    // the forward substitution L u = w
    auto u_row = [&](int i, R (&w)[7]) {
      const R id = (i % 3 == 0) ? idn : idt;
#pragma unroll
      for (int a = 0; a < 6; ++a) w[a] = s2 * R(G[a * NV + i]) * id;
      w[6] = (i % 3 == 0) ? sr * id : R(0);
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        R t = w[a];
#pragma unroll
        for (int k = 0; k < a; ++k) t = fma_r(-L[idx(k, a)], w[k], t);
        w[a] = t * ild[a];
      }
    };
    if (UNROLL && sizeof(R) == 4 && S == 12 && NV <= 24) {  // at most two rows per lane, both formed before either is stored
      R w0[7], w1[7];
      const bool two = lane + 12 < NV;
      u_row(lane < NV ? lane : 0, w0);
      if (two) u_row(lane + 12, w1);
      if (lane < NV)
#pragma unroll
        for (int a = 0; a < 7; ++a) Us[lane * 8 + a] = w0[a];
      if (two)
#pragma unroll
        for (int a = 0; a < 7; ++a) Us[(lane + 12) * 8 + a] = w1[a];
    } else {
      for (int i = lane; i < NV; i += S) {
        R w[7];
        u_row(i, w);
#pragma unroll
        for (int a = 0; a < 7; ++a) Us[i * 8 + a] = w[a];
      }
    }
  }
  __syncthreads();
  // alpha K^-1 = alpha (Dg^-1 - U U^T), entry (i, j) of the upper triangle
  // at Admm<M>::tri(i, j).  Lane p takes the columns j1 = p and
  // j2 = nv-1-p (nv + 1 entries between them; the middle column alone for
  // odd nv), holds their rows of U in registers and walks i = 0 .. j2 in step
  // with the grasp's other lanes: at each i they all read the same row of U,
  // one broadcast load, where spreading single entries over the lanes had
  // each lane read two rows of its own per entry.
  if (active) {
    for (int p = lane; p < (NV + 1) / 2; p += S) {
      const int j1 = p, j2 = NV - 1 - p;
      R u1[7], u2[7];
      load_u_row(Us, j1, u1);
      load_u_row(Us, j2, u2);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (i > j2) break;
        R ui[7];
        load_u_row(Us, i, ui);
        const R di = (i % 3 == 0) ? idn : idt;
        R acc = 0;
#pragma unroll
        for (int a = 0; a < 7; ++a) acc = fma_r(ui[a], u2[a], acc);
        Kinv[Admm<M>::tri(i, j2)] = (float)(R(c.alpha) * ((i == j2 ? di : R(0)) - acc));
        if (i <= j1 && j1 < j2) {
          R acc1 = 0;
#pragma unroll
          for (int a = 0; a < 7; ++a) acc1 = fma_r(ui[a], u1[a], acc1);
          Kinv[Admm<M>::tri(i, j1)] = (float)(R(c.alpha) * ((i == j1 ? di : R(0)) - acc1));
        }
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ ADMM
// One QP per thread.  State: y (nv) and w (nc) with z = Pi(w),
// lam = rho (w - Pi(w)) (Pi: projection onto [l, u]).  With that state the
// OSQP iteration (Stellato et al. 2020, Alg. 1) reads
//   rhs = sigma y - q + rho A^T (2 Pi(w) - w)
//   yt  = K^-1 rhs,   zt = A yt
//   y  <- alpha yt + (1 - alpha) y
//   w  <- w + alpha (zt - Pi(w)).
// The shared memory holds alpha K^-1, so the product below is alpha yt and
// the relaxation costs no separate multiply.
// Row order of A: per contact [f_n, facet 0..7], then the sum row.
// Shared-memory load kept inside the loop that issues it (asm volatile).
// K^-1 is loop-invariant across ADMM iterations; left to itself the
// compiler hoists all of it into registers, which does not fit next to the
// iterate.
__device__ __forceinline__ float lds32(const float* p) {
  float v;
  const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}


__device__ constexpr float kFC[8] = {C8, S8, -S8, -C8, -C8, -S8, S8, C8};
__device__ constexpr float kFS[8] = {S8, C8, C8, S8, -S8, -C8, -C8, -S8};

template <int M>
__device__ __forceinline__ float proj_row(float w, int row, float gamma) {
  // [l, u] per row: f_n in [0, 1], facets in (-inf, 0], sum row in [gamma, inf)
  if (row == 9 * M) return fmaxf(w, gamma);
  if (row % 9 == 0) return fminf(fmaxf(w, 0.f), 1.f);
  return fminf(w, 0.f);
}

// Contribution of one contact's nine rows (v0: the f_n row, vk: the facets)
// to A^T v.  The sum row's entry is added to the normal component by the caller.
// Facets k and k+4 have opposite (d, e) normals (cos, sin of (2k+1) pi/8:
// (C8, S8), (S8, C8), (-S8, C8), (-C8, S8) for k = 0..3), and facets 0, 7
// (1, 6; 2, 5; 3, 4) are mirror images across d: with the pair sums
// s_07 = v_0 + v_7, ... and differences d_07 = v_0 - v_7, ...
//   sum v = (s_07 + s_34) + (s_16 + s_25),
//   d: C8 (s_07 - s_34) + S8 (s_16 - s_25),
//   e: S8 (d_07 + d_34) + C8 (d_16 + d_25)   (d_34 = v_3 - v_4, d_25 = v_2 - v_5).
__device__ __forceinline__ void At_contact(float v0, const float (&vk)[8], float mu_c8, float& gn, float& gd,
                                           float& ge) {
  const float s07 = vk[0] + vk[7], s34 = vk[3] + vk[4], s16 = vk[1] + vk[6], s25 = vk[2] + vk[5];
  const float d07 = vk[0] - vk[7], d34 = vk[3] - vk[4], d16 = vk[1] - vk[6], d25 = vk[2] - vk[5];
  const float sum = (s07 + s34) + (s16 + s25);
  gn = fmaf(-mu_c8, sum, v0);
  gd = fmaf(C8, s07 - s34, S8 * (s16 - s25));
  ge = fmaf(S8, d07 + d34, C8 * (d16 + d25));
}

// Per-contact pieces of one ADMM iteration.  admm_iteration and the
// several-lanes-per-QP form of the batched QP kernel are both written with
// them, so the two give bitwise equal iterates.
// rhs of contact i's three components: sigma y - q + rho A_i^T v with
// v = 2 Pi(w) - w; vsum is the sum row's entry of v.
__device__ __forceinline__ void pyr_contact_rhs(const float* wi, float vsum, const float* yi, const float* mqi,
                                                const AdmmCfg& c, float rho, float* rhs) {
  const float v0 = fmaf(2.f, __saturatef(wi[0]), -wi[0]) + vsum;
  // facet rows (bounds (-inf, 0]): 2 min(w, 0) - w is exactly -|w|, which
  // the hardware applies as a free operand modifier
  float vk[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) vk[k] = -fabsf(wi[1 + k]);
  float gn, gd, ge;
  At_contact(v0, vk, c.mu_c8, gn, gd, ge);
  rhs[0] = fmaf(c.sigma, yi[0], fmaf(rho, gn, mqi[0]));
  rhs[1] = fmaf(c.sigma, yi[1], fmaf(rho, gd, mqi[1]));
  rhs[2] = fmaf(c.sigma, yi[2], fmaf(rho, ge, mqi[2]));
}

// Contact i's nine rows: w <- (w + A_i yt) - alpha Pi(w); (tn, td, te) is
// the contact's part of yt.  On a facet row Pi(w) = min(w, 0) = (w - |w|) / 2,
// so the update is (1 - alpha/2) w + (alpha/2) |w| + (A_i yt)_k: two
// multiply-adds with |w| as a free operand modifier, instead of a min, an
// add and a multiply-add (measured 2.8% faster per fused step).
__device__ __forceinline__ void pyr_contact_update(float* wi, float tn, float td, float te, const AdmmCfg& c) {
  const float al = c.alpha;
  wi[0] = fmaf(-al, __saturatef(wi[0]), wi[0] + tn);
  const float base = -c.mu_c8 * tn;
  const float ka = fmaf(-0.5f, al, 1.f), kb = 0.5f * al;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float zt = fmaf(kFC[k], td, fmaf(kFS[k], te, base));
    wi[1 + k] = fmaf(ka, wi[1 + k], fmaf(kb, fabsf(wi[1 + k]), zt));
  }
}

template <int M>
__device__ __forceinline__ void admm_iteration(float* y, float* w, const float* mq, const float* Kinv,
                                               const AdmmCfg& c, float rho) {
  constexpr int NV = Admm<M>::NV;
  // rhs = sigma y - q + rho A^T v,  v = 2 Pi(w) - w, one contact at a time
  float rhs[NV];
  const float vsum = fmaf(2.f, fmaxf(w[9 * M], c.gamma), -w[9 * M]);
#pragma unroll
  for (int i = 0; i < M; ++i) pyr_contact_rhs(w + 9 * i, vsum, y + 3 * i, mq + 3 * i, c, rho, rhs + 3 * i);
  // yt = alpha K^-1 rhs from the packed upper triangle, column by column:
  // entry (a, b), a <= b, adds K_ab rhs_b to yt_a and, off the diagonal,
  // K_ab rhs_a to yt_b.  The loops unroll completely (every index is a
  // compile-time constant) and each entry is one 4-byte shared load that all
  // lanes of the grasp share.  Measured against row order and against
  // 16-byte loads issued ahead, this order is 2-4% faster per iteration.
  float yt[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) yt[a] = 0.f;
#pragma unroll
  for (int b = 0; b < NV; ++b) {
#pragma unroll
    for (int a = 0; a <= b; ++a) {
      const float kv = lds32(Kinv + Admm<M>::tri(a, b));
      yt[a] = fmaf(kv, rhs[b], yt[a]);
      if (a != b) yt[b] = fmaf(kv, rhs[a], yt[b]);
    }
  }
  // w <- w + alpha (A ys - Pi(w)) = (w + A yt) - alpha Pi(w),
  // y <- alpha ys + (1 - alpha) y = yt + (1 - alpha) y   (yt = alpha ys)
  const float al = c.alpha, bl = 1.0f - c.alpha;
  float sumn = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    sumn += yt[3 * i];
    pyr_contact_update(w + 9 * i, yt[3 * i], yt[3 * i + 1], yt[3 * i + 2], c);
  }
  w[9 * M] = fmaf(-al, fmaxf(w[9 * M], c.gamma), w[9 * M] + sumn);
#pragma unroll
  for (int a = 0; a < NV; ++a) y[a] = fmaf(bl, y[a], yt[a]);
}

// Per-contact pieces of the residuals, shared by admm_residuals and the
// wide form of the batched QP kernel (the maxima do not depend on the order
// in which rows are visited, and every sum is formed in the same order).
// Primal rows of contact i: rp = max(rp, |A_i y - Pi(w_i)|).
template <bool SCALES>
__device__ __forceinline__ void pyr_contact_primal(const float* wi, float yn, float yd, float ye, const AdmmCfg& c,
                                                   float& rp, float& nprim) {
  const float p0 = fminf(fmaxf(wi[0], 0.f), 1.f);
  rp = fmaxf(rp, fabsf(yn - p0));
  if constexpr (SCALES) nprim = fmaxf(nprim, fmaxf(fabsf(yn), fabsf(p0)));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float ay = fmaf(kFC[k], yd, fmaf(kFS[k], ye, -c.mu_c8 * yn));
    const float pk = fminf(wi[1 + k], 0.f);
    rp = fmaxf(rp, fabsf(ay - pk));
    if constexpr (SCALES) nprim = fmaxf(nprim, fmaxf(fabsf(ay), fabsf(pk)));
  }
}

// Contact i's three components of A^T d, d = w - Pi(w) (dsum: the sum row's d).
__device__ __forceinline__ void pyr_contact_atd(const float* wi, float dsum, const AdmmCfg& c, float* at) {
  const float d0 = (wi[0] - fminf(fmaxf(wi[0], 0.f), 1.f)) + dsum;
  float dk[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) dk[k] = wi[1 + k] - fminf(wi[1 + k], 0.f);
  At_contact(d0, dk, c.mu_c8, at[0], at[1], at[2]);
}

// Dual residual of component a: rd = max(rd, |rho (A^T d)_a + (P y)_a + q_a|)
// with P y = 2 G^T (G y) + 2 eps y; gy = G y.  A^T lam = rho A^T d: the sums
// run on d and rho enters once, in an explicit fmaf.
template <int NV, bool SCALES>
__device__ __forceinline__ void dual_component(const float* G, int a, const float* gy, float ya, float mqa, float at,
                                               const AdmmCfg& c, float rho, float& rd, float& ndual) {
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < 6; ++r) s = fmaf(lds32(G + r * NV + a), gy[r], s);
  const float py = fmaf(2.f * c.eps_reg, ya, 2.f * s);
  rd = fmaxf(rd, fabsf(fmaf(rho, at, py - mqa)));
  if constexpr (SCALES) ndual = fmaxf(ndual, fmaxf(fabsf(py), fmaxf(fabsf(rho * at), fabsf(mqa))));
}

// gy = G y (6 x nv, row-major in shared memory), each row summed in column order.
template <int NV>
__device__ __forceinline__ void g_times(const float* G, const float* y, float* gy) {
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < NV; ++a) s = fmaf(lds32(G + r * NV + a), y[a], s);
    gy[r] = s;
  }
}

// Infinity-norm residuals at (y, w): primal |A y - z|, dual |P y + q + A^T lam|,
// z = Pi(w), lam = rho (w - Pi(w)).  With SCALES, also the magnitudes that
// normalise them (OSQP, Stellato et al. 2020, Sec. 5.2):
// scale[0] = max(|A y|, |z|), scale[1] = max(|P y|, |A^T lam|, |q|).
template <int M, bool SCALES = false>
__device__ inline void admm_residuals(const float* y, const float* w, const float* mq, const float* G,
                                      const AdmmCfg& c, float rho, float& rp, float& rd, float* scale = nullptr) {
  constexpr int NV = Admm<M>::NV;
  rp = 0.f;
  float sumn = 0.f, nprim = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    sumn += y[3 * i];
    pyr_contact_primal<SCALES>(w + 9 * i, y[3 * i], y[3 * i + 1], y[3 * i + 2], c, rp, nprim);
  }
  const float psum = fmaxf(w[9 * M], c.gamma);
  rp = fmaxf(rp, fabsf(sumn - psum));
  if constexpr (SCALES) nprim = fmaxf(nprim, fmaxf(fabsf(sumn), fabsf(psum)));
  float gy[6];
  g_times<NV>(G, y, gy);
  const float dsum = w[9 * M] - psum;
  rd = 0.f;
  float ndual = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    float at[3];
    pyr_contact_atd(w + 9 * i, dsum, c, at);
#pragma unroll
    for (int q = 0; q < 3; ++q)
      dual_component<NV, SCALES>(G, 3 * i + q, gy, y[3 * i + q], mq[3 * i + q], at[q], c, rho, rd, ndual);
  }
  if constexpr (SCALES) {
    scale[0] = nprim;
    scale[1] = ndual;
  }
}

// -q = 2 beta G^T t for one wrench t.
template <int M>
__device__ __forceinline__ void neg_q(const float* G, const float* t, float beta, float* mq) {
  constexpr int NV = 3 * M;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 6; ++r) s = fmaf(G[r * NV + a], t[r], s);
    mq[a] = 2.f * beta * s;
  }
}

// ------------------------------------------------------------------ exact QP: nearest point of G C
// With eps_reg = 0 the objective |beta t - G y|^2 depends on y only through
// the wrench G y, so the QP of Eqs. (7)-(9) is the nearest-point problem
// from beta t to the polytope G C in R^6, C the feasible forces.  Wolfe's
// minimum-norm-point algorithm (Wolfe 1976, "Finding the nearest point in a
// polytope", Math. Programming 11) solves it exactly in finitely many steps
// given only a linear-minimisation oracle over C: it keeps the point
// x = G y - beta t as a convex combination of at most 7 points G v_i - beta t
// (v_i vertices of C), adds the oracle's vertex, and moves to the nearest
// point of the affine hull of its set, dropping points whose weight would
// turn negative.
//
// The oracle: minimise g . v over C.  Per contact C is the convex hull of
// the apex 0 and the pyramid's 8 edge tips at f_n = 1,
// E_k = (1, mu cos(k pi/4), mu sin(k pi/4)) in the contact's (n, d, e)
// frame, so contact i contributes c_i f_i with c_i = min_k g_i . E_k and
// f_i in [0, 1] its normal force along its best edge; with sum_i f_i >= gamma
// this is a continuous knapsack: f_i = 1 where c_i < 0, then the cheapest
// remaining contacts filled in order of c_i until the sum reaches gamma.
//
// Stops when the Frank-Wolfe gap |x|^2 - x . q_new (an upper bound on
// Q(y) - Q*) falls to tol max(1, max |q_i|^2), or after max_it oracle calls.
// Returns the oracle calls used (-1: gave up, or stalled on an affinely
// dependent point with a gap above 1e4 tol); y = sum lambda_i v_i and
// Q = |x|^2.  Precision R: double for polishing.
template <int M, typename R>
struct Wolfe {
  static constexpr int NV = 3 * M, K = 8;  // at most 7 points in R^6, one slot for the newcomer
  // v . (oracle) for a gradient gy (in y): the vertex in v, its wrench part G v - b in q
  __device__ static void oracle(const float* G, const R* b, const R* gy, const AdmmCfg& c, R* v, R* q) {
    R cbest[M];
    int kbest[M];
    const R mu = (R)c.mu;
    for (int i = 0; i < M; ++i) {
      R best = 0;
      int kb = 0;
      for (int k = 0; k < 8; ++k) {
        R ck, sk;
        if constexpr (sizeof(R) == 8) sincospi((double)k * 0.25, &sk, &ck);
        else sincospif((float)k * 0.25f, &sk, &ck);
        const R val = gy[3 * i] + mu * (ck * gy[3 * i + 1] + sk * gy[3 * i + 2]);
        if (k == 0 || val < best) best = val, kb = k;
      }
      cbest[i] = best;
      kbest[i] = kb;
    }
    R f[M], sum = 0;
    for (int i = 0; i < M; ++i) {
      f[i] = cbest[i] < 0 ? R(1) : R(0);
      sum += f[i];
    }
    const R gam = (R)c.gamma;
    while (sum < gam) {  // fill the cheapest contact not yet full
      int pick = -1;
      for (int i = 0; i < M; ++i)
        if (f[i] < R(1) && (pick < 0 || cbest[i] < cbest[pick])) pick = i;
      if (pick < 0) break;
      const R add = fmin(R(1) - f[pick], gam - sum);
      f[pick] += add;
      sum += add;
    }
    for (int i = 0; i < M; ++i) {
      R ck, sk;
      if constexpr (sizeof(R) == 8) sincospi((double)kbest[i] * 0.25, &sk, &ck);
      else sincospif((float)kbest[i] * 0.25f, &sk, &ck);
      v[3 * i] = f[i];
      v[3 * i + 1] = f[i] * mu * ck;
      v[3 * i + 2] = f[i] * mu * sk;
    }
    for (int r = 0; r < 6; ++r) {
      R s = -b[r];
      for (int a = 0; a < NV; ++a) s += (R)G[r * NV + a] * v[a];
      q[r] = s;
    }
  }

  __device__ static int solve(const float* G, const float* t, const AdmmCfg& c, const float* y_start, R tol,
                              int max_it, R* y, R& Q) {
    R b[6], V[K][NV], P[K][6], lam[K], x[6], gy[NV];
    for (int r = 0; r < 6; ++r) b[r] = (R)c.beta * (R)t[r];
    // first vertex: the oracle at the gradient of the starting point (any y; zero is fine)
    {
      R ys[NV], res[6];
      for (int a = 0; a < NV; ++a) ys[a] = y_start ? (R)y_start[a] : R(0);
      for (int r = 0; r < 6; ++r) {
        R s = -b[r];
        for (int a = 0; a < NV; ++a) s += (R)G[r * NV + a] * ys[a];
        res[r] = s;
      }
      for (int a = 0; a < NV; ++a) {
        R s = 0;
        for (int r = 0; r < 6; ++r) s += (R)G[r * NV + a] * res[r];
        gy[a] = s;
      }
    }
    oracle(G, b, gy, c, V[0], P[0]);
    int n = 1;
    lam[0] = 1;
    for (int r = 0; r < 6; ++r) x[r] = P[0][r];
    int calls = 1;
    bool ok = true;
    for (;;) {
      // gradient of |x|^2 / 2 in y: G^T x; the oracle's vertex
      for (int a = 0; a < NV; ++a) {
        R s = 0;
        for (int r = 0; r < 6; ++r) s += (R)G[r * NV + a] * x[r];
        gy[a] = s;
      }
      R vn[NV], qn[6];
      oracle(G, b, gy, c, vn, qn);
      ++calls;
      R xx = 0, xq = 0, qmax = 1;
      for (int r = 0; r < 6; ++r) xx += x[r] * x[r], xq += x[r] * qn[r];
      for (int i = 0; i < n; ++i) {
        R s = 0;
        for (int r = 0; r < 6; ++r) s += P[i][r] * P[i][r];
        qmax = fmax(qmax, s);
      }
      if (xx - xq <= tol * qmax) break;  // Frank-Wolfe gap: optimal to tol
      if (calls > max_it || n >= K) return -1;
      for (int a = 0; a < NV; ++a) V[n][a] = vn[a];
      for (int r = 0; r < 6; ++r) P[n][r] = qn[r];
      lam[n++] = 0;
      // minor cycles: nearest point of the affine hull of the set; while it
      // leaves the simplex, step towards it until a weight reaches 0 and drop that point
      for (int guard = 0;; ++guard) {
        if (guard > 2 * K) return -1;
        // affine minimiser: alpha_0 = 1 - sum alpha_i, (D^T D) alpha' = -D^T p_0, D_i = p_i - p_0
        R A[K - 1][K - 1], rhs[K - 1], al[K];
        const int d = n - 1;
        for (int i = 0; i < d; ++i) {
          R s = 0;
          for (int r = 0; r < 6; ++r) s -= (P[i + 1][r] - P[0][r]) * P[0][r];
          rhs[i] = s;
          for (int j = 0; j <= i; ++j) {
            R e = 0;
            for (int r = 0; r < 6; ++r) e += (P[i + 1][r] - P[0][r]) * (P[j + 1][r] - P[0][r]);
            A[i][j] = e;
          }
        }
        bool singular = false;
        for (int j = 0; j < d; ++j) {  // Cholesky, lower triangle in place
          R dd = A[j][j];
          for (int k = 0; k < j; ++k) dd -= A[j][k] * A[j][k];
          if (!(dd > R(sizeof(R) == 8 ? 1e-28 : 1e-14) * qmax)) {
            singular = true;
            break;
          }
          dd = sqrt(dd);
          A[j][j] = dd;
          for (int i = j + 1; i < d; ++i) {
            R s = A[i][j];
            for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
            A[i][j] = s / dd;
          }
        }
        if (singular) {  // the newcomer is affinely dependent on the set: no progress is possible;
          --n;           // the current point stands if its gap is within 1e4 tol
          ok = xx - xq <= R(1e4) * tol * qmax;
          goto done;
        }
        for (int i = 0; i < d; ++i) {
          R s = rhs[i];
          for (int k = 0; k < i; ++k) s -= A[i][k] * rhs[k];
          rhs[i] = s / A[i][i];
        }
        for (int i = d - 1; i >= 0; --i) {
          R s = rhs[i];
          for (int k = i + 1; k < d; ++k) s -= A[k][i] * rhs[k];
          rhs[i] = s / A[i][i];
        }
        R a0 = 1;
        for (int i = 0; i < d; ++i) al[i + 1] = rhs[i], a0 -= rhs[i];
        al[0] = a0;
        bool inside = true;
        for (int i = 0; i < n; ++i) inside = inside && al[i] > 0;
        if (inside) {
          for (int i = 0; i < n; ++i) lam[i] = al[i];
          break;
        }
        R th = 1;  // largest step towards al keeping every weight >= 0
        for (int i = 0; i < n; ++i)
          if (al[i] <= 0) th = fmin(th, lam[i] / (lam[i] - al[i]));
        int w = 0;
        R tot = 0;
        for (int i = 0; i < n; ++i) {
          const R li = lam[i] + th * (al[i] - lam[i]);
          if (li > R(0) && !(al[i] <= 0 && lam[i] / (lam[i] - al[i]) <= th)) {
            lam[w] = li;
            for (int a = 0; a < NV; ++a) V[w][a] = V[i][a];
            for (int r = 0; r < 6; ++r) P[w][r] = P[i][r];
            tot += li;
            ++w;
          }
        }
        n = w;
        for (int i = 0; i < n; ++i) lam[i] /= tot;
        if (n == 1) break;
      }
      for (int r = 0; r < 6; ++r) {
        R s = 0;
        for (int i = 0; i < n; ++i) s += lam[i] * P[i][r];
        x[r] = s;
      }
    }
  done:
    for (int r = 0; r < 6; ++r) {
      R s = 0;
      for (int i = 0; i < n; ++i) s += lam[i] * P[i][r];
      x[r] = s;
    }
    Q = 0;
    for (int r = 0; r < 6; ++r) Q += x[r] * x[r];
    for (int a = 0; a < NV; ++a) {
      R s = 0;
      for (int i = 0; i < n; ++i) s += lam[i] * V[i][a];
      y[a] = s;
    }
    return ok ? calls : -1;
  }
};

// ------------------------------------------------------------------ exact QP in float32
// The same minimum-norm-point method as Wolfe<M, R> (see there), arranged
// for speed in float32: one QP per thread with every array in registers
// (loops fully unrolled over the at most 7 points), the nearest point of the
// affine hull found by a QR factorisation of the differences
// D = [p_1 - p_0, ...] (modified Gram-Schmidt, each column orthogonalised
// twice) instead of the normal equations D^T D, whose float32 conditioning
// (kappa^2) cost accuracy; and vertices held as codes: per contact its best
// edge k (3 bits) and whether it pushes with f = 1 (1 bit), and the one
// contact the knapsack fills fractionally with its f.
// G: the grasp's 6 x 3m matrix (shared memory); b = beta t.  Stops when the
// Frank-Wolfe gap |x|^2 - x . q_new <= 1e-5 |x|^2 + 1e-7 (an upper bound on
// Q(y) - Q*); when the oracle returns a vertex already in the set or one
// affinely dependent on it, or |x|^2 has not fallen by a relative 1e-6 in
// three steps (float32 has no further progress to offer: the point is the
// nearest one at float32 resolution, and its gap bound may then be loose);
// or after max_calls oracle calls.  Returns the calls used,
// negated when the cap stopped it; gap receives the last Frank-Wolfe gap.
template <int M>
struct ExactQP {
  static constexpr int NV = 3 * M, K = 7;
  struct Vtx {
    int code;    // bits 4i..4i+2: contact i's edge k; bit 4i+3: f_i = 1; bits 20..22: fractional contact (7: none)
    float frac;  // the fractional contact's f
  };
  // edge tip directions (1, mu cos(k pi/4), mu sin(k pi/4)): cos, sin of k pi/4
  __device__ static float ck(int k) {
    const float h = 0.70710678118654752f;
    return k == 0 ? 1.f : k == 1 ? h : k == 2 ? 0.f : k == 3 ? -h : k == 4 ? -1.f : k == 5 ? -h : k == 6 ? 0.f : h;
  }
  __device__ static float sk(int k) { return ck((k + 6) & 7); }
  // f_i of contact i in a vertex
  __device__ static float f_of(const Vtx& v, int i) {
    if (((v.code >> 20) & 7) == i) return v.frac;
    return ((v.code >> (4 * i + 3)) & 1) ? 1.f : 0.f;
  }
  // linear oracle: the vertex of C minimising x . (G v) (continuous knapsack
  // over the contacts' best edges), and its point q = G v - b
  __device__ static Vtx oracle(const float* G, const float* b, const float* x, const AdmmCfg& c, float* q) {
    float gy[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) s = fmaf(G[r * NV + a], x[r], s);
      gy[a] = s;
    }
    float cb[M];
    int kb[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      // every multiply-add spelled out: the value must not depend on the
      // code the solve is inlined into (the compiler's contraction does)
      float best = fmaf(c.mu, gy[3 * i + 1], gy[3 * i]);
      int k0 = 0;
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        const float v = fmaf(c.mu, fmaf(ck(k), gy[3 * i + 1], __fmul_rn(sk(k), gy[3 * i + 2])), gy[3 * i]);
        if (v < best) best = v, k0 = k;
      }
      cb[i] = best;
      kb[i] = k0;
    }
    Vtx v;
    v.code = 7 << 20;
    v.frac = 0.f;
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      v.code |= kb[i] << (4 * i);
      if (cb[i] < 0.f) {
        v.code |= 1 << (4 * i + 3);
        sum += 1.f;
      }
    }
    // fill the cheapest contacts not yet at f = 1 until sum f >= gamma
#pragma unroll 1
    for (int guard = 0; guard < M && sum < c.gamma; ++guard) {
      int pick = -1;
      float pc = 0.f;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const bool full = (v.code >> (4 * i + 3)) & 1;
        if (!full && (pick < 0 || cb[i] < pc)) pick = i, pc = cb[i];
      }
      if (pick < 0) break;
      const float add = fminf(1.f, c.gamma - sum);
      if (add >= 1.f) {
        v.code |= 1 << (4 * pick + 3);
      } else {
        v.code = (v.code & ~(7 << 20)) | (pick << 20);
        v.frac = add;  // the fractional contact keeps its 'full' bit clear
      }
      sum += add;
      if (add < 1.f) break;
    }
    point(G, b, v, c, q);
    return v;
  }
  __device__ static void point(const float* G, const float* b, const Vtx& v, const AdmmCfg& c, float* q) {
#pragma unroll
    for (int r = 0; r < 6; ++r) q[r] = -b[r];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const float f = f_of(v, i);
      if (f != 0.f) {
        const int k = (v.code >> (4 * i)) & 7;
        const float fm = __fmul_rn(f, c.mu), fd = __fmul_rn(fm, ck(k)), fe = __fmul_rn(fm, sk(k));
#pragma unroll
        for (int r = 0; r < 6; ++r)
          q[r] = fmaf(f, G[r * NV + 3 * i], fmaf(fd, G[r * NV + 3 * i + 1], fmaf(fe, G[r * NV + 3 * i + 2], q[r])));
      }
    }
  }
  __device__ static void accumulate_y(const Vtx& v, float w, const AdmmCfg& c, float* y) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const float fo = f_of(v, i), f = __fmul_rn(w, fo), fm = __fmul_rn(f, c.mu);
      const int k = (v.code >> (4 * i)) & 7;
      y[3 * i] = fmaf(w, fo, y[3 * i]);
      y[3 * i + 1] = fmaf(fm, ck(k), y[3 * i + 1]);
      y[3 * i + 2] = fmaf(fm, sk(k), y[3 * i + 2]);
    }
  }
  // nearest point of the affine hull of P[0..n-1]: weights al (sum 1);
  // false when the differences are (numerically) dependent.  The loops over
  // the working set run to n, not unrolled to K: the unrolled form missed the
  // instruction cache in the fused step (17% slower there, the same alone)
  __device__ static bool affine_min(const float (&P)[K][6], int n, float (&al)[K]) {
    float U[K - 1][6], R[K - 1][K - 1], sc = 1.f;
#pragma unroll 1
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int r = 0; r < 6; ++r) sc = fmaxf(sc, fabsf(P[i][r]));
#pragma unroll 1
    for (int j = 0; j + 1 < n; ++j) {
      float u[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) u[r] = P[j + 1][r] - P[0][r];
#pragma unroll 1
      for (int i = 0; i < j; ++i) R[i][j] = 0.f;
#pragma unroll
      for (int pass = 0; pass < 2; ++pass)
#pragma unroll 1
        for (int i = 0; i < j; ++i) {
          float d = 0.f;
#pragma unroll
          for (int r = 0; r < 6; ++r) d = fmaf(U[i][r], u[r], d);
          R[i][j] += d;
#pragma unroll
          for (int r = 0; r < 6; ++r) u[r] = fmaf(-d, U[i][r], u[r]);
        }
      float nn = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) nn = fmaf(u[r], u[r], nn);
      const float rjj = sqrtf(nn);
      if (!(rjj > 1e-6f * sc)) return false;
      R[j][j] = rjj;
      const float inv = 1.f / rjj;
#pragma unroll
      for (int r = 0; r < 6; ++r) U[j][r] = u[r] * inv;
    }
    float a1[K - 1];
#pragma unroll 1
    for (int j = n - 2; j >= 0; --j) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) s = fmaf(-U[j][r], P[0][r], s);
#pragma unroll 1
      for (int k = n - 2; k > j; --k) s = fmaf(-R[j][k], a1[k], s);
      a1[j] = s / R[j][j];
    }
    float a0 = 1.f;
#pragma unroll 1
    for (int j = 0; j + 1 < n; ++j) {
      al[j + 1] = a1[j];
      a0 -= a1[j];
    }
    al[0] = a0;
    return true;
  }
  // The working set ("corral"): n points with their vertex codes and weights.
  struct Corral {
    int n;
    Vtx V[K];
    float lam[K];
  };
  // Minor cycles of Wolfe's method on (P, C): the nearest point of the
  // affine hull of the set; while it leaves the simplex, step towards it
  // until a weight reaches 0 and drop that point.  Returns false when the
  // points turned out dependent (the last one is dropped, the weights kept).
  __device__ static bool minor(float (&P)[K][6], Corral& C) {
    int& n = C.n;
#pragma unroll 1
    for (int guard = 0; guard < 2 * K; ++guard) {
      float al[K];
      if (!affine_min(P, n, al)) {  // dependent points: drop the last one, keep the current weights
        --n;
        float tot = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) tot += i < n ? C.lam[i] : 0.f;
        const float it = tot > 0.f ? 1.f / tot : 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) C.lam[i] = i < n ? (tot > 0.f ? C.lam[i] * it : (i == 0 ? 1.f : 0.f)) : 0.f;
        return false;
      }
      bool inside = true;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < n) inside = inside && al[i] > 0.f;
      if (inside) {
#pragma unroll
        for (int i = 0; i < K; ++i) C.lam[i] = i < n ? al[i] : 0.f;
        return true;
      }
      float th = 1.f;
      int drop = -1;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < n && al[i] <= 0.f) {
          const float den = C.lam[i] - al[i];
          const float ti = den > 0.f ? C.lam[i] / den : 0.f;
          if (drop < 0 || ti < th) th = ti, drop = i;
        }
      float tot = 0.f;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < n) {
          C.lam[i] = i == drop ? 0.f : fmaxf(fmaf(th, al[i] - C.lam[i], C.lam[i]), 0.f);
          tot += C.lam[i];
        }
      // compact: move the last point into the dropped slot
      const int last = n - 1;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i == drop && drop != last) {
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j == last) {
              C.V[i] = C.V[j];
              C.lam[i] = C.lam[j];
#pragma unroll
              for (int r = 0; r < 6; ++r) P[i][r] = P[j][r];
            }
        }
      --n;
      const float it = tot > 0.f ? 1.f / tot : 0.f;
#pragma unroll
      for (int i = 0; i < K; ++i) C.lam[i] = i < n ? C.lam[i] * it : 0.f;
      if (n == 1) {
        C.lam[0] = 1.f;
        return true;
      }
    }
    return true;
  }

  // Solves the QP starting from the corral C (C.n == 0: a cold start at the
  // oracle's vertex for y = 0); C receives the final corral, which a later
  // solve of a nearby QP (the next upper step's G) can start from: its
  // points are recomputed for the new G and the minor cycles make it a valid
  // corral again before the first oracle call.
  __device__ static int solve(const float* G, const float* t, const AdmmCfg& c, int max_calls, Corral& C, float* y,
                              float& Q, float& gap) {
    float b[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) b[r] = c.beta * t[r];
    float P[K][6], x[6];
    int calls = 0;
    if (C.n <= 0 || C.n > K) {  // cold: the oracle's vertex at y = 0 (x = -b)
#pragma unroll
      for (int r = 0; r < 6; ++r) x[r] = -b[r];
      C.V[0] = oracle(G, b, x, c, P[0]);
      C.n = 1;
      ++calls;
#pragma unroll
      for (int i = 0; i < K; ++i) C.lam[i] = i == 0 ? 1.f : 0.f;
    } else {  // warm: the stored vertices' points for this G
      float tot = 0.f;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < C.n) {
          point(G, b, C.V[i], c, P[i]);
          C.lam[i] = fmaxf(C.lam[i], 0.f);
          tot += C.lam[i];
        } else {
          C.lam[i] = 0.f;
        }
      const float it = tot > 0.f ? 1.f / tot : 0.f;
#pragma unroll
      for (int i = 0; i < K; ++i) C.lam[i] = i < C.n ? (tot > 0.f ? C.lam[i] * it : 1.f / C.n) : 0.f;
      if (C.n > 1) minor(P, C);
    }
    int& n = C.n;
    bool capped = false;
    int stall = 0;
    float prev_xx = 3.4e38f;
    gap = 0.f;
#pragma unroll 1
    for (;;) {
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i)
          if (i < n) s = fmaf(C.lam[i], P[i][r], s);
        x[r] = s;
      }
      float q[6];
      const Vtx vn = oracle(G, b, x, c, q);
      ++calls;
      float xx = 0.f, xq = 0.f;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        xx = fmaf(x[r], x[r], xx);
        xq = fmaf(x[r], q[r], xq);
      }
      gap = xx - xq;
      if (gap <= fmaf(1e-5f, xx, 1e-7f) || n >= K) break;
      // |x| falls at every major step in exact arithmetic; three steps
      // without a relative 1e-6 decrease: float32 resolution is reached
      stall = xx > prev_xx * (1.f - 1e-6f) ? stall + 1 : 0;
      prev_xx = xx;
      if (stall >= 3) break;
      bool seen = false;  // the oracle cycles back to a vertex of the set
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i < n) seen = seen || (C.V[i].code == vn.code && C.V[i].frac == vn.frac);
      if (seen) break;
      if (calls >= max_calls) {
        capped = true;
        break;
      }
      // add the vertex with weight 0 (slot n), then minor cycles
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (i == n) {
          C.V[i] = vn;
#pragma unroll
          for (int r = 0; r < 6; ++r) P[i][r] = q[r];
          C.lam[i] = 0.f;
        }
      ++n;
      if (!minor(P, C)) {  // the newcomer is dependent: the current point stands
#pragma unroll
        for (int r = 0; r < 6; ++r) {
          float s = 0.f;
#pragma unroll
          for (int i = 0; i < K; ++i)
            if (i < n) s = fmaf(C.lam[i], P[i][r], s);
          x[r] = s;
        }
        break;
      }
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) y[a] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (i < n) accumulate_y(C.V[i], C.lam[i], c, y);
    Q = 0.f;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      float s = c.beta * t[r];
#pragma unroll
      for (int a = 0; a < NV; ++a) s = fmaf(-G[r * NV + a], y[a], s);
      Q = fmaf(s, s, Q);
    }
    return capped ? -calls : calls;
  }
};

// ------------------------------------------------------------------ elliptic cone
// The unlinearised friction model: per contact the row f_n in [0, 1] and
// the cone rows v = (mu f_n, f_d, f_e) in the second-order cone
// {|(v1, v2)| <= v0}; the sum row as before.  Rows: per contact
// [f_n, v0, v1, v2], then the sum row (4m + 1).  The ADMM iteration is the
// pyramid's with this A and the projection onto the cone in the z-update.
constexpr int CONE_PYR = 0, CONE_SOC = 1;

// Euclidean projection onto the second-order cone {|(u1, u2)| <= s}
// (e.g. Parikh & Boyd, Proximal Algorithms, Sec. 6.3.2).
__device__ __forceinline__ void proj_soc(float s, float u1, float u2, float& ps, float& p1, float& p2) {
  const float nu = sqrtf(fmaf(u1, u1, u2 * u2));
  if (nu <= s) {
    ps = s;
    p1 = u1;
    p2 = u2;
  } else if (nu <= -s) {
    ps = p1 = p2 = 0.f;
  } else {  // nu > |s| >= 0
    const float a = 0.5f * (s + nu), k = a / nu;
    ps = a;
    p1 = k * u1;
    p2 = k * u2;
  }
}

// Per-contact pieces of the elliptic-cone iteration (as pyr_contact_rhs /
// pyr_contact_update): rhs of contact i, keeping pc = Pi of its cone rows
// for the update.
__device__ __forceinline__ void soc_contact_rhs(const float* wi, float vsum, const float* yi, const float* mqi,
                                                const AdmmCfg& c, float rho, float* rhs, float* pc) {
  proj_soc(wi[1], wi[2], wi[3], pc[0], pc[1], pc[2]);
  const float v0 = fmaf(2.f, __saturatef(wi[0]), -wi[0]) + vsum;
  const float gn = fmaf(c.mu, fmaf(2.f, pc[0], -wi[1]), v0);
  const float gd = fmaf(2.f, pc[1], -wi[2]), ge = fmaf(2.f, pc[2], -wi[3]);
  rhs[0] = fmaf(c.sigma, yi[0], fmaf(rho, gn, mqi[0]));
  rhs[1] = fmaf(c.sigma, yi[1], fmaf(rho, gd, mqi[1]));
  rhs[2] = fmaf(c.sigma, yi[2], fmaf(rho, ge, mqi[2]));
}

__device__ __forceinline__ void soc_contact_update(float* wi, const float* pc, float tn, float td, float te,
                                                   const AdmmCfg& c) {
  const float al = c.alpha;
  wi[0] = fmaf(-al, __saturatef(wi[0]), wi[0] + tn);
  wi[1] = fmaf(-al, pc[0], fmaf(c.mu, tn, wi[1]));
  wi[2] = fmaf(-al, pc[1], wi[2] + td);
  wi[3] = fmaf(-al, pc[2], wi[3] + te);
}

template <int M>
__device__ __forceinline__ void admm_iteration_soc(float* y, float* w, const float* mq, const float* Kinv,
                                                   const AdmmCfg& c, float rho) {
  constexpr int NV = Admm<M>::NV;
  // rhs = sigma y - q + rho A^T (2 Pi(w) - w), keeping Pi of the cone rows
  float rhs[NV], pc[3 * M];
  const float vsum = fmaf(2.f, fmaxf(w[4 * M], c.gamma), -w[4 * M]);
#pragma unroll
  for (int i = 0; i < M; ++i) soc_contact_rhs(w + 4 * i, vsum, y + 3 * i, mq + 3 * i, c, rho, rhs + 3 * i, pc + 3 * i);
  // yt = alpha K^-1 rhs (packed upper triangle, column order as in admm_iteration)
  float yt[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) yt[a] = 0.f;
#pragma unroll
  for (int b = 0; b < NV; ++b) {
#pragma unroll
    for (int a = 0; a <= b; ++a) {
      const float kv = lds32(Kinv + Admm<M>::tri(a, b));
      yt[a] = fmaf(kv, rhs[b], yt[a]);
      if (a != b) yt[b] = fmaf(kv, rhs[a], yt[b]);
    }
  }
  // w <- (w + A yt) - alpha Pi(w),  y <- yt + (1 - alpha) y   (yt = alpha ys)
  const float al = c.alpha, bl = 1.0f - c.alpha;
  float sumn = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    sumn += yt[3 * i];
    soc_contact_update(w + 4 * i, pc + 3 * i, yt[3 * i], yt[3 * i + 1], yt[3 * i + 2], c);
  }
  w[4 * M] = fmaf(-al, fmaxf(w[4 * M], c.gamma), w[4 * M] + sumn);
#pragma unroll
  for (int a = 0; a < NV; ++a) y[a] = fmaf(bl, y[a], yt[a]);
}

// Primal rows of contact i of the elliptic cone, and d = w - Pi(w) of its
// four rows (per-contact piece of admm_residuals_soc, as pyr_contact_primal).
template <bool SCALES>
__device__ __forceinline__ void soc_contact_primal(const float* wi, float yn, float yd, float ye, const AdmmCfg& c,
                                                   float& rp, float& nprim, float* dl) {
  const float p0 = __saturatef(wi[0]);
  float ps, p1, p2;
  proj_soc(wi[1], wi[2], wi[3], ps, p1, p2);
  rp = fmaxf(rp, fabsf(yn - p0));
  rp = fmaxf(rp, fabsf(fmaf(c.mu, yn, -ps)));
  rp = fmaxf(rp, fabsf(yd - p1));
  rp = fmaxf(rp, fabsf(ye - p2));
  if constexpr (SCALES)
    nprim = fmaxf(fmaxf(nprim, fmaxf(fabsf(yn), fabsf(c.mu * yn))),
                  fmaxf(fmaxf(fabsf(yd), fabsf(ye)), fmaxf(fmaxf(fabsf(p0), fabsf(ps)), fmaxf(fabsf(p1), fabsf(p2)))));
  dl[0] = wi[0] - p0;
  dl[1] = wi[1] - ps;
  dl[2] = wi[2] - p1;
  dl[3] = wi[3] - p2;
}

template <int M, bool SCALES = false>
__device__ inline void admm_residuals_soc(const float* y, const float* w, const float* mq, const float* G,
                                          const AdmmCfg& c, float rho, float& rp, float& rd,
                                          float* scale = nullptr) {
  constexpr int NV = Admm<M>::NV;
  rp = 0.f;
  float sumn = 0.f, nprim = 0.f;
  float dl[4 * M];  // d = w - Pi(w); lam = rho d
#pragma unroll
  for (int i = 0; i < M; ++i) {
    sumn += y[3 * i];
    soc_contact_primal<SCALES>(w + 4 * i, y[3 * i], y[3 * i + 1], y[3 * i + 2], c, rp, nprim, dl + 4 * i);
  }
  const float psum = fmaxf(w[4 * M], c.gamma);
  rp = fmaxf(rp, fabsf(sumn - psum));
  if constexpr (SCALES) nprim = fmaxf(nprim, fmaxf(fabsf(sumn), fabsf(psum)));
  const float dsum = w[4 * M] - psum;
  float ndual = 0.f;
  float gy[6];
  g_times<NV>(G, y, gy);
  rd = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float at[3] = {fmaf(c.mu, dl[4 * i + 1], dl[4 * i]) + dsum, dl[4 * i + 2], dl[4 * i + 3]};
#pragma unroll
    for (int q = 0; q < 3; ++q)
      dual_component<NV, SCALES>(G, 3 * i + q, gy, y[3 * i + q], mq[3 * i + q], at[q], c, rho, rd, ndual);
  }
  if constexpr (SCALES) {
    scale[0] = nprim;
    scale[1] = ndual;
  }
}

// z = Pi(w) of row r of the elliptic-cone rows (the cone rows need the
// whole triple).
template <int M>
__device__ __forceinline__ float proj_row_soc(const float* w, int row, float gamma) {
  if (row == 4 * M) return fmaxf(w[row], gamma);
  const int i = row / 4, k = row % 4;
  if (k == 0) return __saturatef(w[row]);
  float ps, p1, p2;
  proj_soc(w[4 * i + 1], w[4 * i + 2], w[4 * i + 3], ps, p1, p2);
  return k == 1 ? ps : (k == 2 ? p1 : p2);
}

// Runs ADMM on one QP until both residuals are <= eps (checked every
// `check` iterations, eps > 0) or `iters` iterations.  Returns the count
// used; rp/rd receive the last residuals (with eps == 0, computed once at
// the end, and only when want_res: the fused step reports them for its
// last upper step alone).
template <int M, int CONE>
__device__ inline int admm_solve(float* y, float* w, const float* mq, const float* Kinv, const float* G,
                                 const AdmmCfg& c, float& rp, float& rd, bool& conv, bool want_res = true) {
  auto iterate = [&]() {
    if (CONE == CONE_SOC) admm_iteration_soc<M>(y, w, mq, Kinv, c, c.rho);
    else admm_iteration<M>(y, w, mq, Kinv, c, c.rho);
  };
  auto residuals = [&]() {
    if (CONE == CONE_SOC) admm_residuals_soc<M>(y, w, mq, G, c, c.rho, rp, rd);
    else admm_residuals<M>(y, w, mq, G, c, c.rho, rp, rd);
  };
  int it = 0;
  conv = false;
  rp = rd = 0.f;
  if (c.eps > 0.f) {
#pragma unroll 1
    while (it < c.iters) {
      const int chunk = min(c.check, c.iters - it);
#pragma unroll 1
      for (int k = 0; k < chunk; ++k) iterate();
      it += chunk;
      residuals();
      if (rp <= c.eps && rd <= c.eps) {
        conv = true;
        break;
      }
    }
  } else {
#pragma unroll 1
    for (; it < c.iters; ++it) iterate();
    if (want_res) residuals();
  }
  return it;
}

// Re-expresses the iterate for a new penalty rho' (ratio = rho / rho'),
// keeping z = Pi(w) and lam = rho (w - Pi(w)): w <- Pi(w) + ratio (w - Pi(w)).
// Per contact (its rows: f_n and the facets, or f_n and the cone triple) and
// for the sum row; rescale_w and the wide form of the batched QP kernel
// share these.
template <int CONE>
__device__ __forceinline__ void rescale_contact(float* wi, float ratio) {
  if (CONE == CONE_SOC) {
    const float p0 = __saturatef(wi[0]);
    wi[0] = fmaf(ratio, wi[0] - p0, p0);
    float ps, p1, p2;
    proj_soc(wi[1], wi[2], wi[3], ps, p1, p2);
    wi[1] = fmaf(ratio, wi[1] - ps, ps);
    wi[2] = fmaf(ratio, wi[2] - p1, p1);
    wi[3] = fmaf(ratio, wi[3] - p2, p2);
  } else {
    const float p0 = fminf(fmaxf(wi[0], 0.f), 1.f);
    wi[0] = fmaf(ratio, wi[0] - p0, p0);
#pragma unroll
    for (int k = 1; k < 9; ++k) {
      const float p = fminf(wi[k], 0.f);
      wi[k] = fmaf(ratio, wi[k] - p, p);
    }
  }
}
__device__ __forceinline__ float rescale_sum_row(float wsum, float ratio, float gamma) {
  const float p = fmaxf(wsum, gamma);
  return fmaf(ratio, wsum - p, p);
}

template <int M, int CONE>
__device__ inline void rescale_w(float* w, float ratio, const AdmmCfg& c) {
  constexpr int RPC = CONE == CONE_SOC ? 4 : 9;  // rows per contact
#pragma unroll
  for (int i = 0; i < M; ++i) rescale_contact<CONE>(w + RPC * i, ratio);
  w[RPC * M] = rescale_sum_row(w[RPC * M], ratio, c.gamma);
}

// One QP's proposal for log(rho' / rho) in residual balancing (OSQP,
// Stellato et al. 2020, Sec. 5.2): log sqrt((r_p / s_p) / (r_d / s_d)), each
// residual relative to the magnitudes it is formed from (scale of
// admm_residuals).  Unnormalised, a tiny absolute primal residual kept
// pushing rho down to its floor, where the multipliers barely move.
__device__ __forceinline__ float rho_vote(float rp, float rd, const float* scale) {
  return 0.5f * __logf((fmaxf(rp, 1e-12f) * fmaxf(scale[1], 1e-12f)) / (fmaxf(rd, 1e-12f) * fmaxf(scale[0], 1e-12f)));
}

// ADMM to a residual target with the penalty adapted per grasp (the
// residual-balancing rule of OSQP, Stellato et al. 2020, Sec. 5.2):
// every `check` iterations each lane still running proposes
// rho * sqrt((r_p / s_p) / (r_d / s_d)) (rho_vote); when the geometric mean of its grasp's proposals
// moves rho by more than 5x, the grasp re-expresses its iterates and rebuilds
// K^-1 (all of its lanes share one K).  Lanes that converged stop iterating
// but keep their grasp's rho.  Must be called by every thread of the CTA
// (barriers); `active` marks the threads that own a QP, `vote` is S floats
// of shared memory per grasp, `scratch` the K^-1 setup scratch.  c.rho is
// this lane's (its grasp's) current penalty on return.
template <int M, int CONE, typename SetupFn>
__device__ inline int admm_solve_adaptive(bool active, int lane, int S, float* y, float* w, const float* mq,
                                          const float* Kinv, const float* G, AdmmCfg& c, float* vote,
                                          SetupFn&& setup, float& rp, float& rd, bool& conv) {
  int it = 0;
  conv = !active;
  rp = rd = 0.f;
  float scale[2] = {1.f, 1.f};
  const float tol = 1.6094379f;  // log 5
#pragma unroll 1
  for (;;) {
    if (!conv && it < c.iters) {
      const int chunk = min(c.check, c.iters - it);
#pragma unroll 1
      for (int k = 0; k < chunk; ++k) {
        if (CONE == CONE_SOC) admm_iteration_soc<M>(y, w, mq, Kinv, c, c.rho);
        else admm_iteration<M>(y, w, mq, Kinv, c, c.rho);
      }
      it += chunk;
      if (CONE == CONE_SOC) admm_residuals_soc<M, true>(y, w, mq, G, c, c.rho, rp, rd, scale);
      else admm_residuals<M, true>(y, w, mq, G, c, c.rho, rp, rd, scale);
      conv = rp <= c.eps && rd <= c.eps;
    }
    const bool done = conv || it >= c.iters;
    if (__syncthreads_and(done)) break;
    if (active) vote[lane] = done ? 0.f : rho_vote(rp, rd, scale);
    __syncthreads();
    // every lane of a grasp reads the same votes in the same order: one decision per grasp
    float sh = 0.f;
    int cnt = 0;
    if (active)
      for (int j = 0; j < S; ++j) {
        const float v = vote[j];
        sh += v;
        cnt += v != 0.f;
      }
    bool upd = active && cnt > 0 && fabsf(sh / cnt) > tol;
    float rho_new = c.rho;
    if (upd) {
      rho_new = fminf(fmaxf(c.rho * __expf(sh / cnt), 1e-6f), 1e6f);
      upd = rho_new != c.rho;
    }
    // votes read before the next round writes them; no rebuild when no grasp of the CTA moved
    if (!__syncthreads_or(upd)) continue;
    if (upd) {
      rescale_w<M, CONE>(w, c.rho / rho_new, c);
      c.rho = rho_new;
    }
    setup(upd, c);  // rebuilds K^-1 of the grasps that changed (contains barriers)
  }
  return it;
}

// ------------------------------------------------------------------ adjoint
// Envelope-theorem gradient through one contact (Secs. III, IV-A):
// given dE/dG for the contact's three columns (a_k force half, b_k torque
// half, v_k in {n, d, e}):
//   dE/dp = sum_k v_k x b_k,   dE/dv_k = a_k + b_k x p,
// then through the tangent basis d(n), e(n), the normal n = -g/|g| and the
// point p = c - phi g/|g| (g, Hs: SDF gradient and Hessian), plus the
// distance term 2 w_d (phi - alpha - delta) g.  Returns dE/dc.
__device__ inline void contact_adjoint(const ContactGeo& k, const float* dEdG_cols /* [6][3] */,
                                       float dist_coef, float* dEdc) {
  float d[3], e[3];
  tangent_basis(k.n, d, e);
  const float* vk[3] = {k.n, d, e};
  float dEdp[3] = {0.f, 0.f, 0.f};
  float dEdv[3][3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float a[3] = {dEdG_cols[0 * 3 + q], dEdG_cols[1 * 3 + q], dEdG_cols[2 * 3 + q]};
    const float b[3] = {dEdG_cols[3 * 3 + q], dEdG_cols[4 * 3 + q], dEdG_cols[5 * 3 + q]};
    float vb[3], bp[3];
    cross3(vk[q], b, vb);
    cross3(b, k.p, bp);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      dEdp[t] += vb[t];
      dEdv[q][t] = a[t] + bp[t];
    }
  }
  // basis Jacobians (derivative of the Duff construction with the sign fixed)
  const float nx = k.n[0], ny = k.n[1], nz = k.n[2];
  const float sg = copysignf(1.0f, nz);
  const float a = __fdividef(-1.0f, sg + nz);  // as in tangent_basis
  const float a2 = a * a;
  const float Jd[3][3] = {{2.f * sg * nx * a, 0.f, sg * nx * nx * a2},
                          {sg * ny * a, sg * nx * a, sg * nx * ny * a2},
                          {-sg, 0.f, 0.f}};
  const float Je[3][3] = {{ny * a, nx * a, nx * ny * a2}, {0.f, 2.f * ny * a, ny * ny * a2}, {0.f, -1.f, 0.f}};
  float dEdn[3];
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    float s = dEdv[0][cc];
#pragma unroll
    for (int r = 0; r < 3; ++r) s = fmaf(Jd[r][cc], dEdv[1][r], fmaf(Je[r][cc], dEdv[2][r], s));
    dEdn[cc] = s;
  }
  // through p(c), n(c)
  const float iL = rsqrtf(k.g[0] * k.g[0] + k.g[1] * k.g[1] + k.g[2] * k.g[2]);  // as in contact_geometry
  const float no[3] = {k.g[0] * iL, k.g[1] * iL, k.g[2] * iL};
  const float Hs[3][3] = {{k.h[0], k.h[1], k.h[2]}, {k.h[1], k.h[3], k.h[4]}, {k.h[2], k.h[4], k.h[5]}};
  float Dno[3][3];  // (I - no no^T) Hs / L
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) s = fmaf((r == q ? 1.f : 0.f) - no[r] * no[q], Hs[q][cc], s);
      Dno[r][cc] = s * iL;
    }
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float dp = (r == cc ? 1.f : 0.f) - no[r] * k.g[cc] - k.phi * Dno[r][cc];
      s = fmaf(dp, dEdp[r], fmaf(-Dno[r][cc], dEdn[r], s));
    }
    dEdc[cc] = fmaf(dist_coef, k.g[cc], s);
  }
}

// ------------------------------------------------------------------ collision energies
// The constraint energies of Sec. IV-B (joint limits, Eq. (4); no hand-hand /
// hand-object collision) on the hand's collision spheres, cuRobo style:
//   E_pen  = w_pen  sum_k h(r_k + eta_pen - phi(c_k))   (quadratic-then-linear hinge)
//   E_self = w_self sum_pairs max(0, r_a + r_b - |c_a - c_b|)^2
//   E_lim  = w_lim  sum_{k >= 6} max(0, x_k - x_max,k + eta_lim)^2 + max(0, x_min,k + eta_lim - x_k)^2
// and their gradient through the kinematic tree.  The gradient of joint j
// collects, over the links L that joint j moves, the force sum F_L and the
// moment sum tau_L = sum_k c_k x f_k of the sphere gradients f_k = dE/dc_k:
//   dE/dq_j = w_j . (tau - o_j x F),  w_j, o_j: joint j's world axis and point.

__device__ __forceinline__ float penetration_hinge(float p, float eta, float& dh) {
  if (p <= 0.f) {
    dh = 0.f;
    return 0.f;
  }
  if (eta > 0.f && p <= eta) {
    dh = p / eta;
    return 0.5f * p * p / eta;
  }
  dh = 1.f;
  return p - 0.5f * eta;
}

// One grasp's collision energies.  Lanes own slots (links, then the root)
// and joints with stride S.  In (shared memory): frames [12 (n+1)] the link
// and root frames and jw [m][MAXCHAIN][6] the chain joints' world axes and
// points, both from the contact kinematics of this step (every link that
// carries spheres lies on a contact chain).  Scratch: cs [3 K] sphere
// centres; sl [6 (n+1)] per-slot (F, tau), turned into subtree sums in
// place; bw [3 (n+1)] slot bounding-sphere centres.  Out: gc [D] the
// gradient, ep [S] the energy by lane.  Must be called by every thread of
// the CTA (contains barriers).
// The argument structs are copied into registers first: through references
// every use would be a local-memory load that stores to shared memory force
// the compiler to repeat.
static __device__ __noinline__ void collision_phase(bool active, int lane, int S, const HandDev& H, const CollDev& Cr,
                                             const ObjDev& Or, const float* x, const CollParams& Pr,
                                             const float* frames, const float* jw, float* cs, float* sl, float* bw,
                                             float* gc, float* ep) {
  const CollDev C = Cr;
  const ObjDev O = Or;
  const CollParams P = Pr;
  const int n = H.n, D = H.D, nslot = n + 1;
  // a hand without spheres has no sphere tables (null pointers): only the
  // joint-limit term applies.  C.K is uniform, so every thread still meets
  // every barrier below.
  const bool sph = C.K > 0;
  float e = 0.f;
  // C1: sphere centres from the slot frames
  if (active && sph)
    for (int L = lane; L < nslot; L += S) {
      Tf T;
#pragma unroll
      for (int e2 = 0; e2 < 9; ++e2) T.R[e2] = frames[12 * L + e2];
      T.t[0] = frames[12 * L + 9];
      T.t[1] = frames[12 * L + 10];
      T.t[2] = frames[12 * L + 11];
      const int k1 = __ldg(C.slot_start + L + 1);
      for (int k = __ldg(C.slot_start + L); k < k1; ++k) {
        const float4 sp = __ldg(C.sph + k);
        const float p[3] = {sp.x, sp.y, sp.z};
        tf_point(T, p, cs + 3 * k);
      }
      const float4 sb = __ldg(C.sbound + L);
      const float pb[3] = {sb.x, sb.y, sb.z};
      tf_point(T, pb, bw + 3 * L);
    }
  __syncthreads();
  // C2: sphere gradients f_k, summed per slot into (F, tau).  Self pairs:
  // only between slots whose bounding spheres overlap (a mask per slot).
  if (active && sph)
    for (int L = lane; L < nslot; L += S) {
      unsigned long long near = 0ull;
      if (P.w_self != 0.f) {
        const float4 bL = __ldg(C.sbound + L);
        const float cL[3] = {bw[3 * L], bw[3 * L + 1], bw[3 * L + 2]};
        const int q1 = __ldg(C.spstart + L + 1);
        for (int q = __ldg(C.spstart + L); q < q1; ++q) {
          const int L2 = __ldg(C.spartners + q);
          const float dx = cL[0] - bw[3 * L2], dy = cL[1] - bw[3 * L2 + 1], dz = cL[2] - bw[3 * L2 + 2];
          const float rr = bL.w + __ldg(C.sbound + L2).w;
          if (dx * dx + dy * dy + dz * dz < rr * rr) near |= 1ull << L2;
        }
      }
      float F[3] = {0.f, 0.f, 0.f}, tau[3] = {0.f, 0.f, 0.f};
      const int k1 = __ldg(C.slot_start + L + 1);
      for (int k = __ldg(C.slot_start + L); k < k1; ++k) {
        const float c[3] = {cs[3 * k], cs[3 * k + 1], cs[3 * k + 2]};
        const float r = __ldg(C.sph + k).w;
        float f[3] = {0.f, 0.f, 0.f};
        if (P.w_pen != 0.f) {
          const SdfQ q = sdf_query(O, c);
          float dh;
          e = fmaf(P.w_pen, penetration_hinge(r + P.eta_pen - q.phi, P.eta_pen, dh), e);
          const float sc = -P.w_pen * dh;
#pragma unroll
          for (int a = 0; a < 3; ++a) f[a] = sc * q.g[a];
        }
        for (unsigned long long m2 = near; m2; m2 &= m2 - 1ull) {
          const int L2 = __ffsll((long long)m2) - 1;
          const int t1 = __ldg(C.slot_start + L2 + 1);
          for (int o = __ldg(C.slot_start + L2); o < t1; ++o) {
            const float v[3] = {c[0] - cs[3 * o], c[1] - cs[3 * o + 1], c[2] - cs[3 * o + 2]};
            const float len2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            const float rr = r + __ldg(C.sph + o).w;
            if (len2 < rr * rr) {
              const float len = sqrtf(len2);
              const float d = rr - len;
              e = fmaf(0.5f * P.w_self * d, d, e);  // each pair is visited from both spheres
              const float sc = -2.f * P.w_self * d / len;
#pragma unroll
              for (int a = 0; a < 3; ++a) f[a] = fmaf(sc, v[a], f[a]);
            }
          }
        }
        float cf[3];
        cross3(c, f, cf);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F[a] += f[a];
          tau[a] += cf[a];
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sl[6 * L + a] = F[a];
        sl[6 * L + 3 + a] = tau[a];
      }
    }
  __syncthreads();
  // C3a: subtree sums, leaves first (parent[j] < j), by one lane; slot n
  // (the root) becomes the total
  if (active && sph && lane == 0)
    for (int j = n - 1; j >= 0; --j) {
      const int p = H.parent[j];
      const int to = p < 0 ? n : p;
#pragma unroll
      for (int a = 0; a < 6; ++a) sl[6 * to + a] += sl[6 * j + a];
    }
  __syncthreads();
  // C3b: joint gradients dE/dq_j = w_j . (tau_sub - o_j x F_sub) over the
  // links joint j moves (the root joints: everything), and the limit energy
  if (active) {
    for (int k = lane; k < D; k += S) {
      float g = 0.f;
      if (sph) {
        const float* sub = sl + 6 * (k < 6 ? n : k - 6);
        if (k < 3) {
          g = sub[k];
        } else {
          float w[3], o[3];
          if (k < 6) {
            Tf T;
            float om[3][3];
            root_frame(x, T, om);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              w[a] = om[k - 3][a];
              o[a] = x[a];
            }
          } else {
            // joint k-6 on some contact chain (else its subtree has no spheres)
            const float* ax = nullptr;
            for (int i = 0; i < H.m && !ax; ++i)
              if (H.jpos[i][k - 6] >= 0) ax = jw + (i * MAXCHAIN + H.jpos[i][k - 6]) * 6;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              w[a] = ax ? ax[a] : 0.f;
              o[a] = ax ? ax[3 + a] : 0.f;
            }
          }
          const float Fs[3] = {sub[0], sub[1], sub[2]};
          float oF[3];
          cross3(o, Fs, oF);
          g = w[0] * (sub[3] - oF[0]) + w[1] * (sub[4] - oF[1]) + w[2] * (sub[5] - oF[2]);
        }
      }
      if (k >= 6 && P.w_lim != 0.f) {
        const float hi = x[k] - H.qmax[k] + P.eta_lim, lo = H.qmin[k] + P.eta_lim - x[k];
        if (hi > 0.f) {
          e = fmaf(P.w_lim * hi, hi, e);
          g = fmaf(2.f * P.w_lim, hi, g);
        }
        if (lo > 0.f) {
          e = fmaf(P.w_lim * lo, lo, e);
          g = fmaf(-2.f * P.w_lim, lo, g);
        }
      }
      gc[k] = g;
    }
    ep[lane] = e;
  }
  __syncthreads();  // the scratch (fr, cs, sl) is reused by the next phase
}

}  // namespace bodex
