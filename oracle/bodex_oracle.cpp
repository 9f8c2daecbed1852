// BODex coarse-stage inner loop -- plain FP64 CPU ORACLE.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// statement of what the GPU path computes.  Only the test-suite, the smoke
// check and the benchmark's CPU-baseline leg load it; the library under
// paper_2412_16490_gb300/ never does, and the two share no code.
//
// What it computes, in the paper's notation (arXiv 2412.16490):
//   * forward kinematics with a floating base, c_{i,w} = R_i c_{i,l} + T_i
//     (Sec. IV-B), by explicit chain products;
//   * the nearest-point query (Sec. IV-B/IV-C) on an analytic sphere or a
//     node-sampled trilinear SDF: point p_i, inward normal n_i;
//   * the tangent basis (d_i, e_i) with n_i = d_i x e_i and the contact
//     grasp matrix G_i = [n d e; p x n, p x d, p x e] (Sec. III, Eq. (2));
//   * the lower-level QP Q_j (Sec. IV-A, Eqs. (7)-(9)) with the friction
//     cone of Eq. (1) replaced by an inscribed 8-edge pyramid (Sec. IV-A,
//     last paragraph), solved EXACTLY by a primal active-set method
//     (Nocedal & Wright, Numerical Optimization 2nd ed., Alg. 16.3), and by
//     brute-force enumeration of faces for m <= 3 (a second, independent
//     route used to pin the first);
//   * the coarse-stage energy E = w_Q sum_j Q_j + w_d sum_i (phi_i - alpha - delta)^2
//     (Sec. IV-C distance energy, signed, with the 1 cm pre-grasp margin of
//     Sec. IV-D);
//   * its gradient by central differences of E(x) (the definition), and,
//     separately, by the analytic envelope-theorem chain (used by tests);
//   * one Adam step on x followed by clamping to [x_min, x_max] (Eq. (4)).
//
// Readings of points the paper leaves open (beta, gamma, pyramid
// orientation, tangent basis, pose parametrisation, SDF conventions) are
// stated next to the code that takes them.
//
// Build:  g++ -O2 -std=c++17 -ffp-contract=off -shared -fPIC -pthread bodex_oracle.cpp -o libbodex_oracle.so

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

using Vec = std::vector<double>;

// ---------------------------------------------------------------- small 3-vectors
struct V3 {
  double x, y, z;
};
inline V3 v3(const double* a) { return {a[0], a[1], a[2]}; }
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// 3x4 rigid transform [R | t], row-major.
struct Tf {
  double R[9];
  double t[3];
};
Tf tf_identity() {
  Tf T{};
  T.R[0] = T.R[4] = T.R[8] = 1.0;
  return T;
}
Tf tf_mul(const Tf& A, const Tf& B) {
  Tf C{};
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A.R[3 * r + k] * B.R[3 * k + c];
      C.R[3 * r + c] = s;
    }
    double s = A.t[r];
    for (int k = 0; k < 3; ++k) s += A.R[3 * r + k] * B.t[k];
    C.t[r] = s;
  }
  return C;
}
V3 tf_apply(const Tf& T, V3 p) {
  return {T.R[0] * p.x + T.R[1] * p.y + T.R[2] * p.z + T.t[0],
          T.R[3] * p.x + T.R[4] * p.y + T.R[5] * p.z + T.t[1],
          T.R[6] * p.x + T.R[7] * p.y + T.R[8] * p.z + T.t[2]};
}
V3 rot_apply(const double* R, V3 p) {
  return {R[0] * p.x + R[1] * p.y + R[2] * p.z, R[3] * p.x + R[4] * p.y + R[5] * p.z,
          R[6] * p.x + R[7] * p.y + R[8] * p.z};
}
// Rotation by angle q about unit axis a (Rodrigues' formula).
Tf tf_rot(V3 a, double q) {
  const double c = std::cos(q), s = std::sin(q), C = 1.0 - c;
  Tf T{};
  T.R[0] = c + a.x * a.x * C;
  T.R[1] = a.x * a.y * C - a.z * s;
  T.R[2] = a.x * a.z * C + a.y * s;
  T.R[3] = a.y * a.x * C + a.z * s;
  T.R[4] = c + a.y * a.y * C;
  T.R[5] = a.y * a.z * C - a.x * s;
  T.R[6] = a.z * a.x * C - a.y * s;
  T.R[7] = a.z * a.y * C + a.x * s;
  T.R[8] = c + a.z * a.z * C;
  return T;
}
Tf tf_trans(double x, double y, double z) {
  Tf T = tf_identity();
  T.t[0] = x;
  T.t[1] = y;
  T.t[2] = z;
  return T;
}

// ---------------------------------------------------------------- hand and object
struct Hand {
  int n = 0, m = 0, S = 0;
  std::vector<int> parent, clink;
  Vec offset, axis, qmin, qmax, clocal, tips;
  double alpha = 0;
  std::vector<std::vector<char>> anc;  // anc[i][j]: joint j (of 6+n) moves contact i
  // collision spheres: link (-1 = root), centre in the link frame, radius;
  // pairs checked for self-penetration (see build_pairs)
  int K = 0;
  std::vector<int> slink;
  Vec slocal, srad;
  std::vector<std::pair<int, int>> pairs;
};

struct Object {
  int kind = 0;  // 0 = analytic sphere, 1 = node-sampled grid
  V3 center{0, 0, 0};
  double radius = 0;
  int N = 0;
  double h = 0;
  V3 origin{0, 0, 0};
  Vec vals;     // [N^3], index (iz*N + iy)*N + ix
  V3 gc{0, 0, 0};  // gravity centre (origin of the object frame for G)
};

// ---------------------------------------------------------------- forward kinematics
// Pose reading: x = [tx, ty, tz, rx, ry, rz, q_1..q_n] (D = 6 + n).  The
// paper writes x = [r, t, q] with a 9-number rotation (Sec. IV-A) and a
// 6-DoF floating base (Sec. IV-B); the 6-DoF base is taken as three
// prismatic joints along the world axes followed by three revolute joints
// about X, then Y, then Z (intrinsic):  T_root = Trans(t) Rx Ry Rz.
struct FK {
  Tf root;                 // root frame T_root
  std::vector<Tf> T;       // [n] joint frames (after the joint's own rotation)
  std::vector<V3> c;       // [m] contact points in the world
  std::vector<V3> omega;   // [6+n] joint axis in the world (unit, prismatic: direction)
  std::vector<V3> org;     // [6+n] a point on the joint axis in the world
};

FK forward_kinematics(const Hand& H, const double* x) {
  FK out;
  const int n = H.n;
  out.T.resize(n);
  out.omega.resize(6 + n);
  out.org.resize(6 + n);
  const V3 t{x[0], x[1], x[2]};
  const Tf Rx = tf_rot({1, 0, 0}, x[3]);
  const Tf Ry = tf_rot({0, 1, 0}, x[4]);
  const Tf Rz = tf_rot({0, 0, 1}, x[5]);
  const Tf Rxy = tf_mul(Rx, Ry);
  const Tf root = tf_mul(tf_trans(t.x, t.y, t.z), tf_mul(Rxy, Rz));
  out.root = root;
  out.omega[0] = {1, 0, 0};
  out.omega[1] = {0, 1, 0};
  out.omega[2] = {0, 0, 1};
  out.org[0] = out.org[1] = out.org[2] = t;
  out.omega[3] = {1, 0, 0};
  out.omega[4] = rot_apply(Rx.R, {0, 1, 0});
  out.omega[5] = rot_apply(Rxy.R, {0, 0, 1});
  out.org[3] = out.org[4] = out.org[5] = t;
  for (int j = 0; j < n; ++j) {
    const Tf& P = H.parent[j] < 0 ? root : out.T[H.parent[j]];
    Tf off{};
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) off.R[3 * r + c] = H.offset[12 * j + 4 * r + c];
      off.t[r] = H.offset[12 * j + 4 * r + 3];
    }
    const Tf base = tf_mul(P, off);
    const V3 a = v3(&H.axis[3 * j]);
    out.T[j] = tf_mul(base, tf_rot(a, x[6 + j]));
    out.omega[6 + j] = rot_apply(base.R, a);
    out.org[6 + j] = {base.t[0], base.t[1], base.t[2]};
  }
  out.c.resize(H.m);
  for (int i = 0; i < H.m; ++i) out.c[i] = tf_apply(out.T[H.clink[i]], v3(&H.clocal[3 * i]));
  return out;
}

// ---------------------------------------------------------------- SDF query
// phi, its gradient g and Hessian Hs (row-major 3x3) at c, and the voxel cell.
//
// Grid reading: node (ix, iy, iz) holds phi at origin + h*(ix, iy, iz); the
// interpolant is trilinear; cell = floor(u) clamped to [0, N-2] with
// u = (c - origin)/h.  Outside the node box, phi(c) = phi(cl) + |c - cl|
// where cl is c clamped to the box, and g, Hs are the exact derivatives of
// that expression.
struct SdfOut {
  double phi;
  double g[3];
  double Hs[9];
  int cell[3];
};

SdfOut sdf_query(const Object& O, V3 c) {
  SdfOut s{};
  if (O.kind == 0) {
    const V3 v = c - O.center;
    const double L = norm(v);
    s.phi = L - O.radius;
    const V3 u = (1.0 / L) * v;
    const double uu[3] = {u.x, u.y, u.z};
    for (int a = 0; a < 3; ++a) {
      s.g[a] = uu[a];
      for (int b = 0; b < 3; ++b) s.Hs[3 * a + b] = ((a == b ? 1.0 : 0.0) - uu[a] * uu[b]) / L;
    }
    return s;
  }
  const int N = O.N;
  const double h = O.h;
  const double cc[3] = {c.x, c.y, c.z};
  const double org[3] = {O.origin.x, O.origin.y, O.origin.z};
  double cl[3], tt[3];
  bool clamped[3];
  int cell[3];
  for (int a = 0; a < 3; ++a) {
    const double lo = org[a], hi = org[a] + h * (N - 1);
    clamped[a] = cc[a] < lo || cc[a] > hi;
    cl[a] = std::min(std::max(cc[a], lo), hi);
    const double u = (cl[a] - org[a]) / h;
    int k = (int)std::floor(u);
    k = std::min(std::max(k, 0), N - 2);
    cell[a] = k;
    tt[a] = u - k;
  }
  auto val = [&](int ix, int iy, int iz) { return O.vals[((size_t)iz * N + iy) * N + ix]; };
  double phi = 0, gcl[3] = {0, 0, 0}, Hcl[9] = {0};
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const double v = val(cell[0] + cx, cell[1] + cy, cell[2] + cz);
        const double w[3] = {cx ? tt[0] : 1 - tt[0], cy ? tt[1] : 1 - tt[1], cz ? tt[2] : 1 - tt[2]};
        const double dw[3] = {(cx ? 1.0 : -1.0) / h, (cy ? 1.0 : -1.0) / h, (cz ? 1.0 : -1.0) / h};
        phi += w[0] * w[1] * w[2] * v;
        gcl[0] += dw[0] * w[1] * w[2] * v;
        gcl[1] += w[0] * dw[1] * w[2] * v;
        gcl[2] += w[0] * w[1] * dw[2] * v;
        Hcl[1] += dw[0] * dw[1] * w[2] * v;
        Hcl[2] += dw[0] * w[1] * dw[2] * v;
        Hcl[5] += w[0] * dw[1] * dw[2] * v;
      }
  Hcl[3] = Hcl[1];
  Hcl[6] = Hcl[2];
  Hcl[7] = Hcl[5];
  double dv[3], dl2 = 0;
  for (int a = 0; a < 3; ++a) {
    dv[a] = cc[a] - cl[a];
    dl2 += dv[a] * dv[a];
  }
  const double dl = std::sqrt(dl2);
  s.phi = phi + dl;
  for (int a = 0; a < 3; ++a) {
    s.cell[a] = cell[a];
    s.g[a] = clamped[a] ? dv[a] / dl : gcl[a];
    for (int b = 0; b < 3; ++b) {
      double hab = 0;
      if (!clamped[a] && !clamped[b]) hab = Hcl[3 * a + b];
      else if (clamped[a] && clamped[b]) hab = ((a == b ? 1.0 : 0.0) - dv[a] * dv[b] / dl2) / dl;
      s.Hs[3 * a + b] = hab;
    }
  }
  return s;
}

// Nearest-point query (Sec. IV-B): p = c - phi * g/|g|, inward normal n = -g/|g|.
struct Contact {
  V3 p, n;
  double phi;
  SdfOut s;
  bool degenerate;
};
Contact contact_query(const Object& O, V3 c) {
  Contact k{};
  k.s = sdf_query(O, c);
  const V3 g = v3(k.s.g);
  const double L = norm(g);
  k.phi = k.s.phi;
  k.degenerate = !(L >= 1e-12);
  const V3 no = (1.0 / L) * g;
  k.p = c - k.phi * no;
  k.n = -1.0 * no;
  return k;
}

// Tangent basis (d, e) from the unit normal n with n = d x e (Sec. III).
// Reading: the branch-free orthonormal basis of Duff et al., "Building an
// Orthonormal Basis, Revisited", JCGT 6(1), 2017, with sgn = copysign(1, n_z).
void tangent_basis(V3 n, V3* d, V3* e) {
  const double sg = std::copysign(1.0, n.z);
  const double a = -1.0 / (sg + n.z);
  const double b = n.x * n.y * a;
  *d = {1.0 + sg * n.x * n.x * a, sg * b, -sg * n.x};
  *e = {b, sg + n.y * n.y * a, -n.y};
}

// Contact grasp matrix, Sec. III Eq. (2): column block i = [n d e ; p x n, p x d, p x e].
// G is 6 x 3m row-major; p is measured from the object's gravity centre.
void grasp_matrix(int m, const V3* p, const V3* n, V3 gc, double* G) {
  const int nv = 3 * m;
  for (int i = 0; i < m; ++i) {
    V3 d, e;
    tangent_basis(n[i], &d, &e);
    const V3 pr = p[i] - gc;
    const V3 cols[3] = {n[i], d, e};
    for (int k = 0; k < 3; ++k) {
      const V3 tq = cross(pr, cols[k]);
      const int col = 3 * i + k;
      G[0 * nv + col] = cols[k].x;
      G[1 * nv + col] = cols[k].y;
      G[2 * nv + col] = cols[k].z;
      G[3 * nv + col] = tq.x;
      G[4 * nv + col] = tq.y;
      G[5 * nv + col] = tq.z;
    }
  }
}

// ---------------------------------------------------------------- dense linear algebra
// Symmetric eigendecomposition by cyclic Jacobi rotations (Golub & Van Loan,
// Matrix Computations, Sec. 8.5).  A (n x n, row-major) is overwritten; on
// return w holds eigenvalues, V (row-major) the eigenvectors as columns.
void jacobi_eig(int n, Vec A, Vec& w, Vec& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a2 = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += a2;
        if (i != j) off += a2;
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J  (columns p, q)
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A  (rows p, q)
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Householder QR of M (r x c, row-major, r >= c): returns the full orthogonal
// Q (r x r, row-major) and R (c x c upper, row-major).
void householder_qr(int r, int c, const Vec& M, Vec& Q, Vec& R) {
  Vec A = M;
  Q.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) Q[(size_t)i * r + i] = 1.0;
  for (int k = 0; k < c; ++k) {
    double nrm = 0;
    for (int i = k; i < r; ++i) nrm += A[(size_t)i * c + k] * A[(size_t)i * c + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0) continue;
    const double alpha = A[(size_t)k * c + k] > 0 ? -nrm : nrm;
    Vec v(r, 0.0);
    for (int i = k; i < r; ++i) v[i] = A[(size_t)i * c + k];
    v[k] -= alpha;
    double vn = 0;
    for (int i = k; i < r; ++i) vn += v[i] * v[i];
    if (vn == 0) continue;
    for (int j = 0; j < c; ++j) {  // A <- (I - 2vv^T/vn) A
      double s = 0;
      for (int i = k; i < r; ++i) s += v[i] * A[(size_t)i * c + j];
      s *= 2.0 / vn;
      for (int i = k; i < r; ++i) A[(size_t)i * c + j] -= s * v[i];
    }
    for (int i = 0; i < r; ++i) {  // Q <- Q (I - 2vv^T/vn)
      double s = 0;
      for (int l = k; l < r; ++l) s += Q[(size_t)i * r + l] * v[l];
      s *= 2.0 / vn;
      for (int l = k; l < r; ++l) Q[(size_t)i * r + l] -= s * v[l];
    }
  }
  R.assign((size_t)c * c, 0.0);
  for (int i = 0; i < c; ++i)
    for (int j = i; j < c; ++j) R[(size_t)i * c + j] = A[(size_t)i * c + j];
}

// ---------------------------------------------------------------- the lower-level QP
// Sec. IV-A, Eqs. (7)-(9):  Q_j = min_y |beta t_j - G y|^2, y = [f_1..f_m],
// f_i in the friction set of Eq. (1) and sum_i f_{i,1} >= gamma.
// The elliptic cone is replaced by an inscribed pyramid with 8 edges
// (1, mu cos(k pi/4), mu sin(k pi/4)) in the (n, d, e) frame, k = 0..7; its
// facets are  cos(phi_k) f_d + sin(phi_k) f_e <= mu cos(pi/8) f_n  with
// phi_k = (2k+1) pi/8.  Together with 0 <= f_n <= 1 and the sum row.
//
// In "a^T y >= b" form the constraints are numbered, per contact i:
//   10i     : f_n >= 0
//   10i + 1 : -f_n >= -1
//   10i+2+k : mu cos(pi/8) f_n - cos(phi_k) f_d - sin(phi_k) f_e >= 0
// and finally 10m : sum_i f_{i,n} >= gamma.
struct QPProblem {
  int m, nv, nin;
  Vec P;      // nv x nv, objective 1/2 y^T P y + q^T y + const
  Vec q;      // nv
  double c0;  // constant: beta^2 |t|^2
  Vec A;      // nin x nv
  Vec b;      // nin
  Vec G;      // 6 x nv
  Vec w;      // beta t (6)
  double eps = 0;  // optional regulariser eps |y|^2
};

// Rows of the QP constraints A y >= b, per contact: f_n >= 0, -f_n >= -1,
// then K facets mu_f f_n - cos(phi_k) f_d - sin(phi_k) f_e >= 0 with
// phi_k = (2k+1) pi / K; the sum row sum f_n >= gamma last.  The pyramid of
// Sec. IV-A is K = 8 with mu_f = mu cos(pi/8) (inscribed in the cone).
QPProblem make_qp_facets(const double* G, int m, const double* t, double mu_f, int K, double beta, double gamma,
                         double eps_reg) {
  QPProblem Pb;
  Pb.m = m;
  Pb.nv = 3 * m;
  Pb.eps = eps_reg;
  const int nv = Pb.nv, R = 2 + K;
  Pb.nin = R * m + 1;
  Pb.G.assign(G, G + 6 * nv);
  Pb.w.resize(6);
  for (int r = 0; r < 6; ++r) Pb.w[r] = beta * t[r];
  Pb.P.assign((size_t)nv * nv, 0.0);
  Pb.q.assign(nv, 0.0);
  for (int a = 0; a < nv; ++a) {
    for (int b = 0; b < nv; ++b) {
      double s = 0;
      for (int r = 0; r < 6; ++r) s += G[r * nv + a] * G[r * nv + b];
      Pb.P[(size_t)a * nv + b] = 2.0 * s + (a == b ? 2.0 * eps_reg : 0.0);
    }
    double s = 0;
    for (int r = 0; r < 6; ++r) s += G[r * nv + a] * Pb.w[r];
    Pb.q[a] = -2.0 * s;
  }
  Pb.c0 = 0;
  for (int r = 0; r < 6; ++r) Pb.c0 += Pb.w[r] * Pb.w[r];
  Pb.A.assign((size_t)Pb.nin * nv, 0.0);
  Pb.b.assign(Pb.nin, 0.0);
  const double PI = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double* r0 = &Pb.A[(size_t)(R * i) * nv];
    r0[3 * i] = 1.0;
    Pb.b[R * i] = 0.0;
    double* r1 = &Pb.A[(size_t)(R * i + 1) * nv];
    r1[3 * i] = -1.0;
    Pb.b[R * i + 1] = -1.0;
    for (int k = 0; k < K; ++k) {
      const double ph = (2 * k + 1) * PI / K;
      double* rk = &Pb.A[(size_t)(R * i + 2 + k) * nv];
      rk[3 * i] = mu_f;
      rk[3 * i + 1] = -std::cos(ph);
      rk[3 * i + 2] = -std::sin(ph);
      Pb.b[R * i + 2 + k] = 0.0;
    }
  }
  double* rs = &Pb.A[(size_t)(R * m) * nv];
  for (int i = 0; i < m; ++i) rs[3 * i] = 1.0;
  Pb.b[R * m] = gamma;
  return Pb;
}

QPProblem make_qp(const double* G, int m, const double* t, double mu, double beta, double gamma,
                  double eps_reg) {
  const double PI = 3.14159265358979323846;
  return make_qp_facets(G, m, t, mu * std::cos(PI / 8), 8, beta, gamma, eps_reg);
}

double qp_value(const QPProblem& Pb, const double* y) {
  // Q = |beta t - G y|^2 (+ eps |y|^2 when the optional regulariser is on),
  // evaluated directly (not through P, q).  With the regulariser the energy
  // uses the regularised optimal value, whose derivative in G is then the
  // envelope-theorem expression -2 r y^T exactly.
  double Q = 0;
  for (int r = 0; r < 6; ++r) {
    double s = Pb.w[r];
    for (int a = 0; a < Pb.nv; ++a) s -= Pb.G[r * Pb.nv + a] * y[a];
    Q += s * s;
  }
  if (Pb.eps > 0)
    for (int a = 0; a < Pb.nv; ++a) Q += Pb.eps * y[a] * y[a];
  return Q;
}

struct QPResult {
  Vec y;
  Vec lam;                // multipliers of the a^T y >= b rows (0 off the working set)
  std::vector<int> W;     // final working set
  double Q = 0;
  double kkt = 0;         // max of stationarity, infeasibility, dual infeasibility
  int iters = 0;
  int status = 0;         // 0 ok, 1 iteration cap, 2 infeasible parameters
  int unique = 0;         // y* certified unique
};

// One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992): rotates the
// columns of X (r x k, row-major) until they are mutually orthogonal,
// accumulating the rotations in V (k x k, row-major).  On return the
// singular values are the column norms of X.
void one_sided_jacobi(int r, int k, Vec& X, Vec& V) {
  V.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
  double fro = 0;
  for (double v : X) fro += v * v;
  const double tiny = 1e-30 * fro;  // columns this small are numerically zero
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int i = 0; i < k; ++i)
      for (int j = i + 1; j < k; ++j) {
        double a = 0, b = 0, c = 0;
        for (int t = 0; t < r; ++t) {
          const double xi = X[(size_t)t * k + i], xj = X[(size_t)t * k + j];
          a += xi * xi;
          b += xj * xj;
          c += xi * xj;
        }
        if (a <= tiny || b <= tiny || std::fabs(c) <= 1e-15 * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int q = 0; q < r; ++q) {
          const double xi = X[(size_t)q * k + i], xj = X[(size_t)q * k + j];
          X[(size_t)q * k + i] = cs * xi - sn * xj;
          X[(size_t)q * k + j] = sn * xi + cs * xj;
        }
        for (int q = 0; q < k; ++q) {
          const double vi = V[(size_t)q * k + i], vj = V[(size_t)q * k + j];
          V[(size_t)q * k + i] = cs * vi - sn * vj;
          V[(size_t)q * k + j] = sn * vi + cs * vj;
        }
      }
    if (!rotated) break;
  }
}

// Minimise the QP objective over y + Z v (Z: nv x k, row-major).  Because
// P = 2 G^T G (+ 2 eps I) and q = -2 G^T (beta t), the objective is the
// least-squares residual |beta t - G y|^2 (+ eps |y|^2), so on the affine
// set it is  |rhs - M v|^2  with M = G Z, rhs = beta t - G y (and the rows
// sqrt(eps) Z, -sqrt(eps) y when eps > 0).  The minimiser of least norm is
// taken through the SVD of M; working with M rather than Z^T P Z keeps the
// conditioning of G instead of its square.  Returns p = Z v.
void ls_step(const QPProblem& Pb, const Vec& Z, int k, const double* y, double eps_reg, Vec& p) {
  const int nv = Pb.nv;
  p.assign(nv, 0.0);
  if (k == 0) return;
  const int rows = eps_reg > 0 ? 6 + nv : 6;
  Vec X((size_t)rows * k, 0.0), rhs(rows, 0.0);
  for (int r = 0; r < 6; ++r) {
    double s = Pb.w[r];
    for (int a = 0; a < nv; ++a) s -= Pb.G[r * nv + a] * y[a];
    rhs[r] = s;
    for (int j = 0; j < k; ++j) {
      double v = 0;
      for (int a = 0; a < nv; ++a) v += Pb.G[r * nv + a] * Z[(size_t)a * k + j];
      X[(size_t)r * k + j] = v;
    }
  }
  if (eps_reg > 0) {
    const double se = std::sqrt(eps_reg);
    for (int a = 0; a < nv; ++a) {
      rhs[6 + a] = -se * y[a];
      for (int j = 0; j < k; ++j) X[(size_t)(6 + a) * k + j] = se * Z[(size_t)a * k + j];
    }
  }
  Vec V;
  one_sided_jacobi(rows, k, X, V);
  Vec sig(k, 0.0);
  double smax = 0;
  for (int j = 0; j < k; ++j) {
    double s2 = 0;
    for (int r = 0; r < rows; ++r) s2 += X[(size_t)r * k + j] * X[(size_t)r * k + j];
    sig[j] = std::sqrt(s2);
    smax = std::max(smax, sig[j]);
  }
  // Singular values below this are treated as zero curvature: along them
  // the objective's slope is at most 2 tol |rhs|, and a Newton step of
  // (u^T rhs) / sigma would be dominated by rounding.
  const double tol = 1e-10 * std::max(smax, 1.0);
  Vec v(k, 0.0);
  for (int j = 0; j < k; ++j) {
    if (sig[j] <= tol) continue;
    double c = 0;
    for (int r = 0; r < rows; ++r) c += X[(size_t)r * k + j] * rhs[r];
    c /= sig[j] * sig[j];
    for (int i = 0; i < k; ++i) v[i] += c * V[(size_t)i * k + j];
  }
  for (int a = 0; a < nv; ++a) {
    double s = 0;
    for (int j = 0; j < k; ++j) s += Z[(size_t)a * k + j] * v[j];
    p[a] = s;
  }
}

// Null space basis (nv x (nv - |W|)) of the working-set rows, and the QR
// factors of A_W^T for the multiplier solve.
void working_set_factors(const QPProblem& Pb, const std::vector<int>& W, Vec& Z, int& k, Vec& Qf, Vec& Rf) {
  const int nv = Pb.nv, w = (int)W.size();
  Vec AT((size_t)nv * std::max(w, 1), 0.0);
  for (int j = 0; j < w; ++j)
    for (int a = 0; a < nv; ++a) AT[(size_t)a * w + j] = Pb.A[(size_t)W[j] * nv + a];
  if (w == 0) {
    k = nv;
    Z.assign((size_t)nv * nv, 0.0);
    for (int a = 0; a < nv; ++a) Z[(size_t)a * nv + a] = 1.0;
    Qf = Z;
    Rf.clear();
    return;
  }
  householder_qr(nv, w, AT, Qf, Rf);
  k = nv - w;
  Z.assign((size_t)nv * std::max(k, 1), 0.0);
  for (int a = 0; a < nv; ++a)
    for (int j = 0; j < k; ++j) Z[(size_t)a * k + j] = Qf[(size_t)a * nv + (w + j)];
}

// Primal active-set method for the convex QP (Nocedal & Wright Alg. 16.3),
// with the equality-constrained subproblems solved in the null space of the
// working set.  The Hessian P = 2 G^T G is only positive SEMI-definite
// (rank <= 6 < 3m); a zero-curvature descent direction is followed to its
// blocking constraint, which exists because the feasible set is compact.
// Ties among blocking constraints and the choice of the constraint to drop
// follow Bland's lowest-index rule.
QPResult qp_active_set(const QPProblem& Pb) {
  const int nv = Pb.nv, m = Pb.m, nin = Pb.nin;
  QPResult R;
  R.y.assign(nv, 0.0);
  R.lam.assign(nin, 0.0);
  const double gamma = Pb.b[nin - 1];  // the sum row is last
  if (!(gamma <= m) || gamma < 0) {
    R.status = 2;
    return R;
  }
  for (int i = 0; i < m; ++i) R.y[3 * i] = gamma / m;  // feasible start
  std::vector<int> W;
  std::vector<char> inW(nin, 0);
  Vec g(nv), p, Z, Qf, Rf;
  int k = 0;
  for (int it = 0; it < 20000; ++it) {
    R.iters = it + 1;
    for (int a = 0; a < nv; ++a) {
      double s = Pb.q[a];
      for (int b = 0; b < nv; ++b) s += Pb.P[(size_t)a * nv + b] * R.y[b];
      g[a] = s;
    }
    working_set_factors(Pb, W, Z, k, Qf, Rf);
    // Stationary on the working set when the reduced gradient Z^T g vanishes
    // (to rounding); otherwise step toward the subproblem minimiser.
    double gmax = 0, zg = 0;
    for (int a = 0; a < nv; ++a) gmax = std::max(gmax, std::fabs(g[a]));
    for (int j = 0; j < k; ++j) {
      double v = 0;
      for (int a = 0; a < nv; ++a) v += Z[(size_t)a * k + j] * g[a];
      zg = std::max(zg, std::fabs(v));
    }
    bool stationary = zg <= 1e-11 * std::max(1.0, gmax);
    if (!stationary) {
      ls_step(Pb, Z, k, R.y.data(), Pb.eps, p);
      double pm = 0;
      for (int a = 0; a < nv; ++a) pm = std::max(pm, std::fabs(p[a]));
      stationary = pm <= 1e-14;  // at the rounding floor: no step left to take
    }
    double pmax = 0, gp = 0, pPp = 0;
    if (!stationary)
      for (int a = 0; a < nv; ++a) {
        pmax = std::max(pmax, std::fabs(p[a]));
        gp += g[a] * p[a];
        for (int b = 0; b < nv; ++b) pPp += p[a] * Pb.P[(size_t)a * nv + b] * p[b];
      }
    if (stationary || !(gp < 0)) {
      if (!stationary && !(gp < 0)) {
        // The step is not a descent direction (rounding): fall back to the
        // projected steepest-descent direction -Z Z^T g.
        p.assign(nv, 0.0);
        for (int j = 0; j < k; ++j) {
          double v = 0;
          for (int a = 0; a < nv; ++a) v += Z[(size_t)a * k + j] * g[a];
          for (int a = 0; a < nv; ++a) p[a] -= Z[(size_t)a * k + j] * v;
        }
        pmax = gp = pPp = 0;
        for (int a = 0; a < nv; ++a) {
          pmax = std::max(pmax, std::fabs(p[a]));
          gp += g[a] * p[a];
          for (int b = 0; b < nv; ++b) pPp += p[a] * Pb.P[(size_t)a * nv + b] * p[b];
        }
      }
    }
    if (stationary) {
      // multipliers: A_W^T lam = g
      const int w = (int)W.size();
      Vec lamW(w, 0.0);
      if (w > 0) {
        Vec rhs(w, 0.0);
        for (int j = 0; j < w; ++j) {
          double s = 0;
          for (int a = 0; a < nv; ++a) s += Qf[(size_t)a * nv + j] * g[a];
          rhs[j] = s;
        }
        for (int j = w - 1; j >= 0; --j) {
          double s = rhs[j];
          for (int l = j + 1; l < w; ++l) s -= Rf[(size_t)j * w + l] * lamW[l];
          lamW[j] = s / Rf[(size_t)j * w + j];
        }
      }
      int drop = -1;
      for (int j = 0; j < w; ++j)
        if (lamW[j] < -1e-12 && (drop < 0 || W[j] < W[drop])) drop = j;
      if (drop < 0) {
        std::fill(R.lam.begin(), R.lam.end(), 0.0);
        for (int j = 0; j < w; ++j) R.lam[W[j]] = lamW[j];
        break;
      }
      inW[W[drop]] = 0;
      W.erase(W.begin() + drop);
      continue;
    }
    // Ratio test.  A row counts as blocking only if p decreases it by more
    // than rounding (relative to |p|): rows in the span of the working set
    // have a^T p = 0 exactly in exact arithmetic and must not be added.
    // Exact line search along p (the objective is quadratic), capped by the
    // ratio test; the least-squares step has its minimiser at 1.
    double step = pPp > 0 ? -gp / pPp : std::numeric_limits<double>::infinity();
    int block = -1;
    const double aptol = 1e-11 * std::max(pmax, 1e-300);
    for (int i = 0; i < nin; ++i) {
      if (inW[i]) continue;
      double ap = 0, ay = 0;
      for (int a = 0; a < nv; ++a) {
        ap += Pb.A[(size_t)i * nv + a] * p[a];
        ay += Pb.A[(size_t)i * nv + a] * R.y[a];
      }
      if (ap < -aptol) {
        const double si = std::max(0.0, (Pb.b[i] - ay) / ap);
        if (si < step) {
          step = si;
          block = i;
        }
      }
    }
    if (!std::isfinite(step)) {  // zero curvature and nothing blocks: impossible on a bounded set
      R.status = 3;
      break;
    }
    for (int a = 0; a < nv; ++a) R.y[a] += step * p[a];
    if (block >= 0) {
      W.push_back(block);
      inW[block] = 1;
    }
  }
  if (R.iters >= 20000 && R.status == 0) R.status = 1;
  R.W = W;
  R.Q = qp_value(Pb, R.y.data());
  // KKT certificate: stationarity, primal feasibility, dual feasibility,
  // complementarity.
  double kkt = 0;
  for (int a = 0; a < nv; ++a) {
    double s = Pb.q[a];
    for (int b = 0; b < nv; ++b) s += Pb.P[(size_t)a * nv + b] * R.y[b];
    for (int i = 0; i < nin; ++i) s -= R.lam[i] * Pb.A[(size_t)i * nv + a];
    kkt = std::max(kkt, std::fabs(s));
  }
  for (int i = 0; i < nin; ++i) {
    double ay = -Pb.b[i];
    for (int a = 0; a < nv; ++a) ay += Pb.A[(size_t)i * nv + a] * R.y[a];
    kkt = std::max(kkt, std::max(0.0, -ay));
    kkt = std::max(kkt, std::max(0.0, -R.lam[i]));
    kkt = std::max(kkt, std::fabs(R.lam[i] * ay));
  }
  R.kkt = kkt;
  // Uniqueness of y*: strict complementarity on every active row, and the
  // stacked matrix [G; A_active] has a trivial null space.
  bool strict = true;
  std::vector<int> act;
  for (int i = 0; i < nin; ++i) {
    double ay = -Pb.b[i];
    for (int a = 0; a < nv; ++a) ay += Pb.A[(size_t)i * nv + a] * R.y[a];
    if (std::fabs(ay) < 1e-9) {
      act.push_back(i);
      if (!(R.lam[i] > 1e-9)) strict = false;
    }
  }
  const int rows = 6 + (int)act.size();
  Vec MtM((size_t)nv * nv, 0.0);
  for (int a = 0; a < nv; ++a)
    for (int b = 0; b < nv; ++b) {
      double s = 0;
      for (int r = 0; r < 6; ++r) s += Pb.G[r * nv + a] * Pb.G[r * nv + b];
      for (int i : act) s += Pb.A[(size_t)i * nv + a] * Pb.A[(size_t)i * nv + b];
      MtM[(size_t)a * nv + b] = s;
    }
  (void)rows;
  Vec ew, EV;
  jacobi_eig(nv, MtM, ew, EV);
  double emin = 1e300, emax = 0;
  for (double v : ew) {
    emin = std::min(emin, v);
    emax = std::max(emax, v);
  }
  R.unique = (strict && emin > 1e-10 * std::max(1.0, emax)) ? 1 : 0;
  if (Pb.eps > 0) R.unique = 1;  // eps |y|^2 makes the objective strictly convex
  return R;
}

// Brute force over the faces of the feasible set, m <= 3 (used to pin the
// active-set solver).  Each contact's truncated octagonal pyramid has 35
// faces: its relative interior, 8 side facets, the cap f_n = 1, 8 side
// edges, 8 cap edges, 8 cap vertices and the apex f = 0; the sum row is
// either active or not.  On every face's affine hull the least-norm
// minimiser is computed; the optimum is the smallest objective among the
// minimisers that are feasible (a vertex of the optimal set is the unique
// minimiser on the affine hull of the face that holds it).
double qp_bruteforce(const QPProblem& Pb, Vec* ybest) {
  const int m = Pb.m, nv = Pb.nv;
  // face f of one contact -> list of rows (local index into the 10-row block;
  // 100 + c means the coordinate row y_c = 0 used for the apex)
  std::vector<std::vector<int>> faces;
  faces.push_back({});
  for (int k = 0; k < 8; ++k) faces.push_back({2 + k});
  faces.push_back({1});
  for (int k = 0; k < 8; ++k) faces.push_back({2 + k, 2 + (k + 1) % 8});
  for (int k = 0; k < 8; ++k) faces.push_back({2 + k, 1});
  for (int k = 0; k < 8; ++k) faces.push_back({2 + k, 2 + (k + 1) % 8, 1});
  faces.push_back({100, 101, 102});
  const int F = (int)faces.size();
  long total = 1;
  for (int i = 0; i < m; ++i) total *= F;
  double best = std::numeric_limits<double>::infinity();
  Vec E, bE, y(nv);
  for (long code = 0; code < total; ++code) {
    for (int sumact = 0; sumact < 2; ++sumact) {
      E.clear();
      bE.clear();
      long c = code;
      for (int i = 0; i < m; ++i) {
        const auto& fc = faces[c % F];
        c /= F;
        for (int r : fc) {
          Vec row(nv, 0.0);
          double rhs = 0;
          if (r >= 100) {
            row[3 * i + (r - 100)] = 1.0;
          } else {
            for (int a = 0; a < nv; ++a) row[a] = Pb.A[(size_t)(10 * i + r) * nv + a];
            rhs = Pb.b[10 * i + r];
          }
          E.insert(E.end(), row.begin(), row.end());
          bE.push_back(rhs);
        }
      }
      if (sumact) {
        for (int a = 0; a < nv; ++a) E.push_back(Pb.A[(size_t)(10 * m) * nv + a]);
        bE.push_back(Pb.b[10 * m]);
      }
      const int ne = (int)bE.size();
      if (ne > nv) continue;
      // least-norm particular solution and null space via QR of E^T
      Vec Z;
      int k;
      Vec y0(nv, 0.0);
      if (ne > 0) {
        Vec ET((size_t)nv * ne);
        for (int j = 0; j < ne; ++j)
          for (int a = 0; a < nv; ++a) ET[(size_t)a * ne + j] = E[(size_t)j * nv + a];
        Vec Qf, Rf;
        householder_qr(nv, ne, ET, Qf, Rf);
        bool singular = false;
        for (int j = 0; j < ne; ++j)
          if (std::fabs(Rf[(size_t)j * ne + j]) < 1e-12) singular = true;
        if (singular) continue;
        Vec s(ne);
        for (int j = 0; j < ne; ++j) {  // R^T s = b
          double v = bE[j];
          for (int l = 0; l < j; ++l) v -= Rf[(size_t)l * ne + j] * s[l];
          s[j] = v / Rf[(size_t)j * ne + j];
        }
        for (int a = 0; a < nv; ++a) {
          double v = 0;
          for (int j = 0; j < ne; ++j) v += Qf[(size_t)a * nv + j] * s[j];
          y0[a] = v;
        }
        k = nv - ne;
        Z.assign((size_t)nv * std::max(k, 1), 0.0);
        for (int a = 0; a < nv; ++a)
          for (int j = 0; j < k; ++j) Z[(size_t)a * k + j] = Qf[(size_t)a * nv + ne + j];
      } else {
        k = nv;
        Z.assign((size_t)nv * nv, 0.0);
        for (int a = 0; a < nv; ++a) Z[(size_t)a * nv + a] = 1.0;
      }
      Vec p;
      ls_step(Pb, Z, k, y0.data(), Pb.eps, p);
      for (int a = 0; a < nv; ++a) y[a] = y0[a] + p[a];
      bool feas = true;
      for (int i = 0; i < Pb.nin && feas; ++i) {
        double ay = 0;
        for (int a = 0; a < nv; ++a) ay += Pb.A[(size_t)i * nv + a] * y[a];
        if (ay < Pb.b[i] - 1e-9) feas = false;
      }
      if (!feas) continue;
      const double Q = qp_value(Pb, y.data());
      if (Q < best) {
        best = Q;
        if (ybest) *ybest = y;
      }
    }
  }
  return best;
}

// ---------------------------------------------------------------- energy and gradient
// energy: 0 = the QP grasp energy (Eqs. (7)-(9)); 1 = the DFC force-closure
// energy of Liu et al. 2021 (the comparison of Sec. V-C), see dfc_wrench.
struct Params {
  double mu, beta, gamma, w_q, w_d, delta, eps_reg, lr_t, lr_r, b1, b2, adam_eps;
  int energy;
  double w_pen, w_self, w_lim, eta_pen, eta_lim;  // collision energies (collision_energy)
  int cone;         // 0: the 8-facet pyramid; 1: the elliptic cone (qp_soc, inscribed bound)
  int cone_facets;  // K of qp_soc
};
Params params_from(const double* a) {
  return {a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], a[8], a[9], a[10], a[11], (int)a[12],
          a[13], a[14], a[15], a[16], a[17], (int)a[18], (int)a[19]};
}

// DFC (Liu et al. 2021) assumes frictionless contacts that all push with the
// same unit force along the inward normal; the grasp is force closure when
// the resulting net wrench vanishes.  Its energy is |w|^2 with
//   w = sum_i [n_i; p_i x n_i] = G u,  u = 1 on every normal component.
void dfc_wrench(const Vec& G, int m, double w[6]) {
  const int nv = 3 * m;
  for (int r = 0; r < 6; ++r) {
    w[r] = 0;
    for (int i = 0; i < m; ++i) w[r] += G[r * nv + 3 * i];
  }
}

struct Eval {
  Vec x;
  FK fk;
  std::vector<Contact> ct;
  Vec G;
  std::vector<QPResult> qp;
  double E = 0;
  int status = 0;
};

// E(x) = w_Q sum_j Q_j + w_d sum_i (phi_i - alpha - delta)^2.
// Distance-energy reading: the paper's coarse term is (|c - p| - alpha)^2
// (Sec. IV-C); the signed SDF value replaces |c - p| so that penetration is
// penalised, and delta is the pre-grasp margin (Sec. IV-D).
// ---------------------------------------------------------------- elliptic friction cone
// The unlinearised contact model (Sec. III, the paper's Eqs. before the
// pyramid of Sec. IV-A): each force in the elliptic cone |(f_d, f_e)| <=
// mu f_n with 0 <= f_n <= 1, plus sum f_n >= gamma -- a second-order-cone
// program.  Its optimum Q* is bracketed by two exact polyhedral QPs: the
// K-facet pyramid inscribed in the cone (facet distance mu cos(pi/K)) gives
// Q_in >= Q* with a point y_in that is feasible for the cone, and the
// circumscribed one (facet distance mu) gives Q_out <= Q*.  The bracket
// closes as 1 - cos(pi/K).  Multipliers in the GPU's row form (per contact
// the f_n row, then the cone rows (mu f_n, f_d, f_e); then the sum row)
// come from the inscribed solve: the facets' combine into a point of the
// polar cone.
struct SocResult {
  Vec y, lam;  // y = y_in; lam: 4m + 1 rows
  double Q_in = 0, Q_out = 0, kkt = 0;
  int status = 0;  // 0 ok, 1 an active-set solve hit its cap, 2 infeasible parameters
};

SocResult qp_soc(const double* G, int m, const double* t6, double mu, double beta, double gamma, double eps_reg,
                 int K) {
  const double PI = 3.14159265358979323846;
  SocResult R;
  QPProblem Pin = make_qp_facets(G, m, t6, mu * std::cos(PI / K), K, beta, gamma, eps_reg);
  QPProblem Pout = make_qp_facets(G, m, t6, mu, K, beta, gamma, eps_reg);
  QPResult Ri = qp_active_set(Pin), Ro = qp_active_set(Pout);
  R.y = Ri.y;
  R.Q_in = Ri.Q;
  R.Q_out = Ro.Q;
  R.kkt = std::max(Ri.kkt, Ro.kkt);
  R.status = std::max(Ri.status, Ro.status);
  R.lam.assign(4 * m + 1, 0.0);
  const int rows = 2 + K;
  const double mf = mu * std::cos(PI / K);
  for (int i = 0; i < m; ++i) {
    // A y >= b rows with multiplier l >= 0 enter grad f = sum l a; the row
    // form has grad f + A_row^T lam = 0, so lam = -(the rows' combination)
    R.lam[4 * i] = Ri.lam[rows * i + 1] - Ri.lam[rows * i];  // f_n <= 1 (upper) minus f_n >= 0 (lower)
    double v0 = 0, v1 = 0, v2 = 0;
    for (int k = 0; k < K; ++k) {
      const double l = Ri.lam[rows * i + 2 + k], ph = (2 * k + 1) * PI / K;
      v0 += l * mf / mu;
      v1 -= l * std::cos(ph);
      v2 -= l * std::sin(ph);
    }
    R.lam[4 * i + 1] = -v0;
    R.lam[4 * i + 2] = -v1;
    R.lam[4 * i + 3] = -v2;
  }
  R.lam[4 * m] = -Ri.lam[rows * m];
  return R;
}

// ---------------------------------------------------------------- collision energies
// The constraints of Eq. (4) (joint limits) and "no hand-hand / hand-object
// collision", as cuRobo-style energies on the hand's collision spheres
// (Sec. IV-B).  Readings:
//   penetration  E_pen  = w_pen sum_s h(r_s + eta_pen - phi(c_s)), with the
//                h(p) = 0 (p <= 0), p^2 / (2 eta) (0 < p <= eta), p - eta/2
//                (p > eta), a quadratic-then-linear hinge (eta = 0: max(p, 0));
//   self         E_self = w_self sum_{(a,b) in pairs} max(0, r_a + r_b - |c_a - c_b|)^2;
//   joint limits E_lim  = w_lim sum_{k >= 6} max(0, x_k - x_max,k + eta_lim)^2
//                                          + max(0, x_min,k + eta_lim - x_k)^2.
// Pairs: spheres on different links, except a link and its nearest
// ancestor link that carries spheres (the root counts as such an ancestor),
// which touch by construction (neighbouring links).
void build_pairs(Hand& H) {
  std::vector<char> has(H.n, 0);
  for (int s = 0; s < H.K; ++s)
    if (H.slink[s] >= 0) has[H.slink[s]] = 1;
  auto eff_parent = [&](int L) {  // -1: the root; -2: none (L is the root)
    if (L < 0) return -2;
    int p = H.parent[L];
    while (p >= 0 && !has[p]) p = H.parent[p];
    return p;
  };
  H.pairs.clear();
  for (int a = 0; a < H.K; ++a)
    for (int b = a + 1; b < H.K; ++b) {
      const int la = H.slink[a], lb = H.slink[b];
      if (la == lb || eff_parent(la) == lb || eff_parent(lb) == la) continue;
      H.pairs.emplace_back(a, b);
    }
}

bool moves(const Hand& H, int jx, int link) {  // does joint jx (of 6+n) move `link`?
  if (jx < 6) return true;
  for (int j = link; j >= 0; j = H.parent[j])
    if (j == jx - 6) return true;
  return false;
}

double penetration_hinge(double p, double eta, double* dh) {
  if (p <= 0) {
    *dh = 0;
    return 0;
  }
  if (eta > 0 && p <= eta) {
    *dh = p / eta;
    return p * p / (2 * eta);
  }
  *dh = 1;
  return p - 0.5 * eta;
}

// E_pen + E_self + E_lim at x (frames f); adds the gradient to g when given.
double collision_energy(const Hand& H, const Object& O, const FK& f, const double* x, const Params& P, double* g) {
  const int D = 6 + H.n;
  double E = 0;
  std::vector<V3> c(H.K), dc(H.K, V3{0, 0, 0});
  for (int s = 0; s < H.K; ++s)
    c[s] = tf_apply(H.slink[s] < 0 ? f.root : f.T[H.slink[s]], v3(&H.slocal[3 * s]));
  if (P.w_pen != 0)
    for (int s = 0; s < H.K; ++s) {
      const SdfOut q = sdf_query(O, c[s]);
      double dh;
      E += P.w_pen * penetration_hinge(H.srad[s] + P.eta_pen - q.phi, P.eta_pen, &dh);
      dc[s] = dc[s] - (P.w_pen * dh) * V3{q.g[0], q.g[1], q.g[2]};
    }
  if (P.w_self != 0)
    for (const auto& pr : H.pairs) {
      const V3 v = c[pr.first] - c[pr.second];
      const double L = std::sqrt(dot(v, v));
      const double d = H.srad[pr.first] + H.srad[pr.second] - L;
      if (d <= 0) continue;
      E += P.w_self * d * d;
      const V3 u = (1.0 / L) * v;
      dc[pr.first] = dc[pr.first] - (2 * P.w_self * d) * u;
      dc[pr.second] = dc[pr.second] + (2 * P.w_self * d) * u;
    }
  if (P.w_lim != 0)
    for (int k = 6; k < D; ++k) {
      const double hi = x[k] - H.qmax[k] + P.eta_lim, lo = H.qmin[k] + P.eta_lim - x[k];
      if (hi > 0) {
        E += P.w_lim * hi * hi;
        if (g) g[k] += 2 * P.w_lim * hi;
      }
      if (lo > 0) {
        E += P.w_lim * lo * lo;
        if (g) g[k] -= 2 * P.w_lim * lo;
      }
    }
  if (g)
    for (int s = 0; s < H.K; ++s)
      for (int jx = 0; jx < D; ++jx) {
        if (!moves(H, jx, H.slink[s])) continue;
        const V3 d = jx < 3 ? f.omega[jx] : cross(f.omega[jx], c[s] - f.org[jx]);
        g[jx] += dot(dc[s], d);
      }
  return E;
}

bool has_collision_terms(const Params& P) { return P.w_pen != 0 || P.w_self != 0 || P.w_lim != 0; }

Eval evaluate(const Hand& H, const Object& O, const double* x, const Params& P, const double* T, int s) {
  Eval ev;
  ev.x.assign(x, x + 6 + H.n);
  ev.fk = forward_kinematics(H, x);
  const int m = H.m;
  ev.ct.resize(m);
  std::vector<V3> p(m), n(m);
  double Ed = 0;
  for (int i = 0; i < m; ++i) {
    ev.ct[i] = contact_query(O, ev.fk.c[i]);
    if (ev.ct[i].degenerate) ev.status = 1;
    p[i] = ev.ct[i].p;
    n[i] = ev.ct[i].n;
    const double r = ev.ct[i].phi - H.alpha - P.delta;
    Ed += r * r;
  }
  ev.G.assign(6 * 3 * m, 0.0);
  grasp_matrix(m, p.data(), n.data(), O.gc, ev.G.data());
  double EQ = 0;
  if (P.energy == 1) {
    double w[6];
    dfc_wrench(ev.G, m, w);
    for (int r = 0; r < 6; ++r) EQ += w[r] * w[r];
  } else if (P.cone == 1) {  // Q_j from the inscribed K-facet pyramid (within 1 - cos(pi/K) of the cone)
    ev.qp.resize(s);
    for (int j = 0; j < s; ++j) {
      SocResult R = qp_soc(ev.G.data(), m, T + 6 * j, P.mu, P.beta, P.gamma, P.eps_reg, P.cone_facets);
      ev.qp[j].y = R.y;
      ev.qp[j].Q = R.Q_in;
      ev.qp[j].status = R.status;
      EQ += R.Q_in;
    }
  } else {
    ev.qp.resize(s);
    for (int j = 0; j < s; ++j) {
      QPProblem Pb = make_qp(ev.G.data(), m, T + 6 * j, P.mu, P.beta, P.gamma, P.eps_reg);
      ev.qp[j] = qp_active_set(Pb);
      EQ += ev.qp[j].Q;
    }
  }
  ev.E = P.w_q * EQ + P.w_d * Ed;
  if (has_collision_terms(P)) ev.E += collision_energy(H, O, ev.fk, x, P, nullptr);
  return ev;
}

double energy(const Hand& H, const Object& O, const double* x, const Params& P, const double* T, int s) {
  return evaluate(H, O, x, P, T, s).E;
}

// Gradient by FP64 central differences of E(x), step h.
void grad_fd(const Hand& H, const Object& O, const double* x, const Params& P, const double* T, int s, double h,
             double* g) {
  const int D = 6 + H.n;
  Vec xp(x, x + D);
  for (int k = 0; k < D; ++k) {
    xp[k] = x[k] + h;
    const double ep = energy(H, O, xp.data(), P, T, s);
    xp[k] = x[k] - h;
    const double em = energy(H, O, xp.data(), P, T, s);
    xp[k] = x[k];
    g[k] = (ep - em) / (2.0 * h);
  }
}

// Analytic gradient (second, independent route; tests pin it against grad_fd).
// Envelope theorem (Danskin): the feasible set of Eq. (7)-(9) does not depend
// on x, so dQ_j/dG = -2 r_j y_j^T with r_j = beta t_j - G y_j at the optimum.
void grad_analytic(const Hand& H, const Object& O, const Eval& ev, const Params& P, const double* T, int s,
                   double* g) {
  const int m = H.m, nv = 3 * m, D = 6 + H.n;
  Vec dG(6 * nv, 0.0);
  if (P.energy == 1) {  // d|G u|^2 / dG = 2 (G u) u^T
    double w[6];
    dfc_wrench(ev.G, m, w);
    for (int r = 0; r < 6; ++r)
      for (int i = 0; i < m; ++i) dG[r * nv + 3 * i] = 2.0 * P.w_q * w[r];
  }
  for (int j = 0; j < (P.energy == 1 ? 0 : s); ++j) {
    const Vec& y = ev.qp[j].y;
    for (int r = 0; r < 6; ++r) {
      double rr = P.beta * T[6 * j + r];
      for (int a = 0; a < nv; ++a) rr -= ev.G[r * nv + a] * y[a];
      for (int a = 0; a < nv; ++a) dG[r * nv + a] += -2.0 * P.w_q * rr * y[a];
    }
  }
  std::fill(g, g + D, 0.0);
  for (int i = 0; i < m; ++i) {
    const Contact& ct = ev.ct[i];
    V3 d, e;
    tangent_basis(ct.n, &d, &e);
    const V3 pr = ct.p - O.gc;
    const V3 vk[3] = {ct.n, d, e};
    V3 dEdp{0, 0, 0}, dEdv[3];
    for (int k = 0; k < 3; ++k) {
      const int col = 3 * i + k;
      const V3 a{dG[0 * nv + col], dG[1 * nv + col], dG[2 * nv + col]};
      const V3 b{dG[3 * nv + col], dG[4 * nv + col], dG[5 * nv + col]};
      dEdp = dEdp + cross(vk[k], b);
      dEdv[k] = a + cross(b, pr);
    }
    // through the tangent basis d(n), e(n)
    const V3 n = ct.n;
    const double sg = std::copysign(1.0, n.z);
    const double a = -1.0 / (sg + n.z);
    const double a2 = a * a;
    // Jacobians J[r][c] = d(vec_r)/d(n_c)
    const double Jd[3][3] = {{2 * sg * n.x * a, 0, sg * n.x * n.x * a2},
                             {sg * n.y * a, sg * n.x * a, sg * n.x * n.y * a2},
                             {-sg, 0, 0}};
    const double Je[3][3] = {{n.y * a, n.x * a, n.x * n.y * a2}, {0, 2 * n.y * a, n.y * n.y * a2}, {0, -1, 0}};
    double dEdn[3] = {dEdv[0].x, dEdv[0].y, dEdv[0].z};
    const double gd[3] = {dEdv[1].x, dEdv[1].y, dEdv[1].z}, ge[3] = {dEdv[2].x, dEdv[2].y, dEdv[2].z};
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) dEdn[c] += Jd[r][c] * gd[r] + Je[r][c] * ge[r];
    // through p(c), n(c):  n_out = g/|g|, n = -n_out, p = c - phi n_out
    const double* gs = ct.s.g;
    const double* Hs = ct.s.Hs;
    const double L = std::sqrt(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
    double no[3] = {gs[0] / L, gs[1] / L, gs[2] / L};
    double Dno[3][3];  // d n_out / d c = (I - no no^T) Hs / L
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double v = 0;
        for (int k = 0; k < 3; ++k) v += ((r == k ? 1.0 : 0.0) - no[r] * no[k]) * Hs[3 * k + c];
        Dno[r][c] = v / L;
      }
    const double gp[3] = {dEdp.x, dEdp.y, dEdp.z};
    double dEdc[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      double v = 0;
      for (int r = 0; r < 3; ++r) {
        const double dp = (r == c ? 1.0 : 0.0) - no[r] * gs[c] - ct.phi * Dno[r][c];
        const double dn = -Dno[r][c];
        v += dp * gp[r] + dn * dEdn[r];
      }
      v += 2.0 * P.w_d * (ct.phi - H.alpha - P.delta) * gs[c];
      dEdc[c] = v;
    }
    // through forward kinematics
    const V3 gc{dEdc[0], dEdc[1], dEdc[2]};
    const V3 ci = ev.fk.c[i];
    for (int jx = 0; jx < D; ++jx) {
      if (!H.anc[i][jx]) continue;
      V3 dc;
      if (jx < 3) dc = ev.fk.omega[jx];
      else dc = cross(ev.fk.omega[jx], ci - ev.fk.org[jx]);
      g[jx] += dot(gc, dc);
    }
  }
  if (has_collision_terms(P)) collision_energy(H, O, ev.fk, ev.x.data(), P, g);
}

// One Adam step (Kingma & Ba 2015) on x, then clamp to [x_min, x_max]
// (Eq. (4)).  Learning rate lr_t for the three translations, lr_r for all
// angles.  t is the 1-based step count.
void adam_step(const Hand& H, const Params& P, double* x, double* mm, double* vv, const double* g, int t) {
  const int D = 6 + H.n;
  const double c1 = 1.0 - std::pow(P.b1, t), c2 = 1.0 - std::pow(P.b2, t);
  for (int k = 0; k < D; ++k) {
    mm[k] = P.b1 * mm[k] + (1.0 - P.b1) * g[k];
    vv[k] = P.b2 * vv[k] + (1.0 - P.b2) * g[k] * g[k];
    const double mh = mm[k] / c1, vh = vv[k] / c2;
    const double lr = k < 3 ? P.lr_t : P.lr_r;
    x[k] -= lr * mh / (std::sqrt(vh) + P.adam_eps);
    x[k] = std::min(std::max(x[k], H.qmin[k]), H.qmax[k]);
  }
}

void build_ancestors(Hand& H) {
  const int D = 6 + H.n;
  H.anc.assign(H.m, std::vector<char>(D, 0));
  for (int i = 0; i < H.m; ++i) {
    for (int k = 0; k < 6; ++k) H.anc[i][k] = 1;
    for (int j = H.clink[i]; j >= 0; j = H.parent[j]) H.anc[i][6 + j] = 1;
  }
}

// ---------------------------------------------------------------- refinement (fine / final stages)
// Sec. IV-C, Eqs. (10)-(11), in SDF form.  The fingertip surface of contact
// i is a fixed set of S sample points s_{i,k} in its link frame.  Reading:
//   c^f_i   = the sample with the smallest phi (lowest k on ties),
//   p^f_i   = its nearest object point, c^f - phi n_out,
//   c^{f'}  = R_i Detach(s_{i,k*}) + T_i  (equals c^f; only R_i, T_i vary),
//   E^f     = w_d sum_i |c^{f'}_i - (p^f_i + delta n_out,i)|^2
//           + w_qp sum_i |c^{f'}_i - p^c_i|^2,
// p^f and the margin target are constants (not differentiated), p^c are the
// object points at the end of the coarse stage.  delta = 1 cm in the fine
// stage (pre-grasp, Sec. IV-D) and 0 in the final stage, where the first
// term is the paper's |c^{f'} - p^f|^2.
struct Refine {
  double E = 0;
  std::vector<int> kstar;
  std::vector<double> gap;  // phi(second best) - phi(best), for tie detection
};

Tf link_frame(const FK& f, const Hand& H, int i) { return f.T[H.clink[i]]; }

Refine refine_eval(const Hand& H, const Object& O, const double* x, const double* pc, double delta, double w_d,
                   double w_qp, double* g) {
  Refine R;
  const int D = 6 + H.n;
  FK f = forward_kinematics(H, x);
  R.kstar.assign(H.m, 0);
  R.gap.assign(H.m, 0.0);
  if (g) std::fill(g, g + D, 0.0);
  for (int i = 0; i < H.m; ++i) {
    const Tf T = link_frame(f, H, i);
    double best = std::numeric_limits<double>::infinity(), second = best;
    int kb = 0;
    for (int k = 0; k < H.S; ++k) {
      const V3 ck = tf_apply(T, v3(&H.tips[((size_t)i * H.S + k) * 3]));
      const double ph = sdf_query(O, ck).phi;
      if (ph < best) {
        second = best;
        best = ph;
        kb = k;
      } else if (ph < second) {
        second = ph;
      }
    }
    R.kstar[i] = kb;
    R.gap[i] = second - best;
    const V3 cf = tf_apply(T, v3(&H.tips[((size_t)i * H.S + kb) * 3]));
    const Contact ct = contact_query(O, cf);
    const V3 target = ct.p - delta * ct.n;  // p^f + delta n_out (n is inward)
    const V3 pci = v3(pc + 3 * i);
    const V3 a = cf - target, b = cf - pci;
    R.E += w_d * dot(a, a) + w_qp * dot(b, b);
    if (!g) continue;
    const V3 dEdc = 2.0 * w_d * a + 2.0 * w_qp * b;
    for (int jx = 0; jx < D; ++jx) {
      if (!H.anc[i][jx]) continue;
      const V3 dc = jx < 3 ? f.omega[jx] : cross(f.omega[jx], cf - f.org[jx]);
      g[jx] += dot(dEdc, dc);
    }
  }
  return R;
}

// Contact Distance Consistency (Sec. V-B): the spread between the largest
// and the smallest signed fingertip distance over the m fingers.  A
// fingertip's signed distance is the smallest phi over its surface samples
// (the fine-stage reading of the fingertip surface); a hand without samples
// uses its coarse sphere, phi(c_i) - alpha.
struct Metrics {
  std::vector<double> d;
  double cdc = 0;
};

Metrics contact_metrics(const Hand& H, const Object& O, const double* x) {
  Metrics R;
  FK f = forward_kinematics(H, x);
  R.d.assign(H.m, 0.0);
  for (int i = 0; i < H.m; ++i) {
    if (H.S > 0) {
      const Tf T = link_frame(f, H, i);
      double best = std::numeric_limits<double>::infinity();
      for (int k = 0; k < H.S; ++k)
        best = std::min(best, sdf_query(O, tf_apply(T, v3(&H.tips[((size_t)i * H.S + k) * 3]))).phi);
      R.d[i] = best;
    } else {
      R.d[i] = sdf_query(O, f.c[i]).phi - H.alpha;
    }
  }
  if (H.m > 0) {
    const auto mm = std::minmax_element(R.d.begin(), R.d.end());
    R.cdc = *mm.second - *mm.first;
  }
  return R;
}

template <class F>
void parallel_for(int count, int threads, F&& f) {
  threads = std::max(1, std::min(threads, count));
  if (threads == 1) {
    for (int i = 0; i < count; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t)
    pool.emplace_back([&, t] {
      for (int i = t; i < count; i += threads) f(i);
    });
  for (auto& th : pool) th.join();
}

}  // namespace

// ============================================================================ C interface (ctypes)
extern "C" {

void* orc_hand_new(int n, int m, const int32_t* parent, const float* offset, const float* axis, const float* qmin,
                   const float* qmax, const int32_t* clink, const float* clocal, double alpha, int S,
                   const float* tips, int K, const int32_t* slink, const float* slocal, const float* srad) {
  Hand* H = new Hand();
  H->n = n;
  H->m = m;
  H->S = S;
  H->parent.assign(parent, parent + n);
  H->clink.assign(clink, clink + m);
  H->offset.assign(offset, offset + 12 * n);
  H->axis.assign(axis, axis + 3 * n);
  H->qmin.assign(qmin, qmin + 6 + n);
  H->qmax.assign(qmax, qmax + 6 + n);
  H->clocal.assign(clocal, clocal + 3 * m);
  if (S > 0 && tips) H->tips.assign(tips, tips + 3 * (size_t)m * S);
  H->alpha = alpha;
  build_ancestors(*H);
  H->K = (K > 0 && slink && slocal && srad) ? K : 0;
  if (H->K > 0) {
    H->slink.assign(slink, slink + K);
    H->slocal.assign(slocal, slocal + 3 * (size_t)K);
    H->srad.assign(srad, srad + K);
  }
  build_pairs(*H);
  return H;
}
void orc_hand_free(void* h) { delete static_cast<Hand*>(h); }

void* orc_object_sphere(double cx, double cy, double cz, double r) {
  Object* O = new Object();
  O->kind = 0;
  O->center = {cx, cy, cz};
  O->radius = r;
  O->gc = O->center;  // gravity centre of a solid sphere
  return O;
}

// Gravity-centre reading for a grid: the FP64 mean position of the nodes
// whose sampled value is negative (inside the object).
void* orc_object_grid(int N, double h, const float* origin, const float* vals) {
  Object* O = new Object();
  O->kind = 1;
  O->N = N;
  O->h = h;
  O->origin = {origin[0], origin[1], origin[2]};
  O->vals.assign(vals, vals + (size_t)N * N * N);
  double sx = 0, sy = 0, sz = 0;
  long cnt = 0;
  for (int iz = 0; iz < N; ++iz)
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix)
        if (O->vals[((size_t)iz * N + iy) * N + ix] < 0) {
          sx += O->origin.x + h * ix;
          sy += O->origin.y + h * iy;
          sz += O->origin.z + h * iz;
          ++cnt;
        }
  if (cnt > 0) O->gc = {sx / cnt, sy / cnt, sz / cnt};
  else O->gc = {O->origin.x + h * (N - 1) / 2, O->origin.y + h * (N - 1) / 2, O->origin.z + h * (N - 1) / 2};
  return O;
}
void orc_object_free(void* o) { delete static_cast<Object*>(o); }
void orc_object_gc(void* o, double* gc) {
  const Object* O = static_cast<Object*>(o);
  gc[0] = O->gc.x;
  gc[1] = O->gc.y;
  gc[2] = O->gc.z;
}

// FK for B poses: contact points c [B,m,3], joint world axes / origins [B,6+n,3].
void orc_fk(void* h, const double* x, int B, double* c, double* omega, double* org) {
  const Hand& H = *static_cast<Hand*>(h);
  const int D = 6 + H.n;
  for (int b = 0; b < B; ++b) {
    FK f = forward_kinematics(H, x + (size_t)b * D);
    for (int i = 0; i < H.m; ++i) {
      c[((size_t)b * H.m + i) * 3 + 0] = f.c[i].x;
      c[((size_t)b * H.m + i) * 3 + 1] = f.c[i].y;
      c[((size_t)b * H.m + i) * 3 + 2] = f.c[i].z;
    }
    if (omega)
      for (int j = 0; j < D; ++j) {
        omega[((size_t)b * D + j) * 3 + 0] = f.omega[j].x;
        omega[((size_t)b * D + j) * 3 + 1] = f.omega[j].y;
        omega[((size_t)b * D + j) * 3 + 2] = f.omega[j].z;
        org[((size_t)b * D + j) * 3 + 0] = f.org[j].x;
        org[((size_t)b * D + j) * 3 + 1] = f.org[j].y;
        org[((size_t)b * D + j) * 3 + 2] = f.org[j].z;
      }
  }
}

// Link frames of all joints [B,n,12] (row-major 3x4), for FK pins.
void orc_fk_frames(void* h, const double* x, int B, double* frames) {
  const Hand& H = *static_cast<Hand*>(h);
  const int D = 6 + H.n;
  for (int b = 0; b < B; ++b) {
    FK f = forward_kinematics(H, x + (size_t)b * D);
    for (int j = 0; j < H.n; ++j)
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) frames[((size_t)b * H.n + j) * 12 + 4 * r + c] = f.T[j].R[3 * r + c];
        frames[((size_t)b * H.n + j) * 12 + 4 * r + 3] = f.T[j].t[r];
      }
  }
}

// SDF query for K points: phi [K], grad [K,3], hess [K,9], cell [K,3].
void orc_sdf(void* o, const double* c, int K, double* phi, double* grad, double* hess, int32_t* cell) {
  const Object& O = *static_cast<Object*>(o);
  for (int k = 0; k < K; ++k) {
    SdfOut s = sdf_query(O, v3(c + 3 * k));
    phi[k] = s.phi;
    for (int a = 0; a < 3; ++a) {
      grad[3 * k + a] = s.g[a];
      cell[3 * k + a] = s.cell[a];
    }
    for (int a = 0; a < 9; ++a) hess[9 * k + a] = s.Hs[a];
  }
}

// Nearest-point query for K points: p [K,3], inward normal n [K,3], phi [K].
void orc_contact(void* o, const double* c, int K, double* p, double* n, double* phi, int32_t* degenerate) {
  const Object& O = *static_cast<Object*>(o);
  for (int k = 0; k < K; ++k) {
    Contact ct = contact_query(O, v3(c + 3 * k));
    p[3 * k] = ct.p.x;
    p[3 * k + 1] = ct.p.y;
    p[3 * k + 2] = ct.p.z;
    n[3 * k] = ct.n.x;
    n[3 * k + 1] = ct.n.y;
    n[3 * k + 2] = ct.n.z;
    phi[k] = ct.phi;
    degenerate[k] = ct.degenerate ? 1 : 0;
  }
}

void orc_basis(const double* n, int K, double* d, double* e) {
  for (int k = 0; k < K; ++k) {
    V3 dd, ee;
    tangent_basis(v3(n + 3 * k), &dd, &ee);
    d[3 * k] = dd.x;
    d[3 * k + 1] = dd.y;
    d[3 * k + 2] = dd.z;
    e[3 * k] = ee.x;
    e[3 * k + 1] = ee.y;
    e[3 * k + 2] = ee.z;
  }
}

// G [B,6,3m] from p, n [B,m,3] and the gravity centre gc [3].
void orc_grasp_matrix(const double* p, const double* n, int B, int m, const double* gc, double* G) {
  std::vector<V3> pp(m), nn(m);
  for (int b = 0; b < B; ++b) {
    for (int i = 0; i < m; ++i) {
      pp[i] = v3(p + ((size_t)b * m + i) * 3);
      nn[i] = v3(n + ((size_t)b * m + i) * 3);
    }
    grasp_matrix(m, pp.data(), nn.data(), v3(gc), G + (size_t)b * 18 * m);
  }
}

// Exact QP solves for B grasps x s wrenches.  G [B,6,3m], T [s,6].
// Outputs: y [B,s,3m], Q [B,s], kkt [B,s], unique [B,s], status [B,s],
// lam [B,s,10m+1] (may be NULL), iters [B,s] (may be NULL).
void orc_qp_solve(const double* G, int B, int m, const double* T, int s, double mu, double beta, double gamma,
                  double eps_reg, int threads, double* y, double* Q, double* kkt, int32_t* unique, int32_t* status,
                  double* lam, int32_t* iters) {
  const int nv = 3 * m, nin = 10 * m + 1;
  parallel_for(B * s, threads, [&](int idx) {
    const int b = idx / s, j = idx % s;
    QPProblem Pb = make_qp(G + (size_t)b * 6 * nv, m, T + 6 * j, mu, beta, gamma, eps_reg);
    QPResult R = qp_active_set(Pb);
    std::copy(R.y.begin(), R.y.end(), y + (size_t)idx * nv);
    Q[idx] = R.Q;
    kkt[idx] = R.kkt;
    unique[idx] = R.unique;
    status[idx] = R.status;
    if (lam) std::copy(R.lam.begin(), R.lam.end(), lam + (size_t)idx * nin);
    if (iters) iters[idx] = R.iters;
  });
}

// Elliptic-cone problems (qp_soc, K facets per bracketing pyramid) for B x s
// wrenches: y [B,s,3m] (the inscribed optimum), Q_in, Q_out [B,s], kkt,
// status [B,s], lam [B,s,4m+1] (may be NULL).
void orc_qp_soc(const double* G, int B, int m, const double* T, int s, double mu, double beta, double gamma,
                double eps_reg, int K, int threads, double* y, double* Q_in, double* Q_out, double* kkt,
                int32_t* status, double* lam) {
  const int nv = 3 * m;
  parallel_for(B * s, threads, [&](int idx) {
    const int b = idx / s, j = idx % s;
    SocResult R = qp_soc(G + (size_t)b * 6 * nv, m, T + 6 * j, mu, beta, gamma, eps_reg, K);
    std::copy(R.y.begin(), R.y.end(), y + (size_t)idx * nv);
    Q_in[idx] = R.Q_in;
    Q_out[idx] = R.Q_out;
    kkt[idx] = R.kkt;
    status[idx] = R.status;
    if (lam) std::copy(R.lam.begin(), R.lam.end(), lam + (size_t)idx * (4 * m + 1));
  });
}

// Brute-force optimum (m <= 3) for B x s problems: Q [B,s], y [B,s,3m].
void orc_qp_bruteforce(const double* G, int B, int m, const double* T, int s, double mu, double beta, double gamma,
                       double eps_reg, int threads, double* Q, double* y) {
  const int nv = 3 * m;
  parallel_for(B * s, threads, [&](int idx) {
    const int b = idx / s, j = idx % s;
    QPProblem Pb = make_qp(G + (size_t)b * 6 * nv, m, T + 6 * j, mu, beta, gamma, eps_reg);
    Vec yb;
    Q[idx] = qp_bruteforce(Pb, &yb);
    if (y && !yb.empty()) std::copy(yb.begin(), yb.end(), y + (size_t)idx * nv);
  });
}

// Full evaluation at B poses.  Outputs (any may be NULL except E):
//   E [B], c [B,m,3], p [B,m,3], n [B,m,3], phi [B,m], cell [B,m,3], G [B,6,3m],
//   Q [B,s], y [B,s,3m], unique [B,s], grad_a [B,D] (analytic), status [B].
void orc_evaluate(void* h, void* o, const double* x, int B, const double* params, const double* T, int s,
                  int threads, double* E, double* c, double* p, double* n, double* phi, int32_t* cell, double* G,
                  double* Q, double* y, int32_t* unique, double* grad_a, int32_t* status) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const Params P = params_from(params);
  const int m = H.m, nv = 3 * m, D = 6 + H.n;
  parallel_for(B, threads, [&](int b) {
    Eval ev = evaluate(H, O, x + (size_t)b * D, P, T, s);
    E[b] = ev.E;
    if (status) status[b] = ev.status;
    for (int i = 0; i < m; ++i) {
      const size_t o3 = ((size_t)b * m + i) * 3;
      const V3 cc = ev.fk.c[i], pp = ev.ct[i].p, nn = ev.ct[i].n;
      if (c) { c[o3] = cc.x; c[o3 + 1] = cc.y; c[o3 + 2] = cc.z; }
      if (p) { p[o3] = pp.x; p[o3 + 1] = pp.y; p[o3 + 2] = pp.z; }
      if (n) { n[o3] = nn.x; n[o3 + 1] = nn.y; n[o3 + 2] = nn.z; }
      if (phi) phi[(size_t)b * m + i] = ev.ct[i].phi;
      if (cell) for (int a = 0; a < 3; ++a) cell[o3 + a] = ev.ct[i].s.cell[a];
    }
    if (G) std::copy(ev.G.begin(), ev.G.end(), G + (size_t)b * 6 * nv);
    for (int j = 0; j < (int)ev.qp.size(); ++j) {  // no QPs under the DFC energy
      if (Q) Q[(size_t)b * s + j] = ev.qp[j].Q;
      if (y) std::copy(ev.qp[j].y.begin(), ev.qp[j].y.end(), y + ((size_t)b * s + j) * nv);
      if (unique) unique[(size_t)b * s + j] = ev.qp[j].unique;
    }
    if (grad_a) grad_analytic(H, O, ev, P, T, s, grad_a + (size_t)b * D);
  });
}

// Central-difference gradient of E at B poses: grad [B,D].
void orc_grad_fd(void* h, void* o, const double* x, int B, const double* params, const double* T, int s, double step,
                 int threads, double* grad) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const Params P = params_from(params);
  const int D = 6 + H.n;
  parallel_for(B, threads, [&](int b) { grad_fd(H, O, x + (size_t)b * D, P, T, s, step, grad + (size_t)b * D); });
}

// Adam + clamp for B poses given gradients (t = 1-based step count).
void orc_adam(void* h, const double* params, double* x, double* mm, double* vv, const double* grad, int B, int t) {
  const Hand& H = *static_cast<Hand*>(h);
  const Params P = params_from(params);
  const int D = 6 + H.n;
  for (int b = 0; b < B; ++b)
    adam_step(H, P, x + (size_t)b * D, mm + (size_t)b * D, vv + (size_t)b * D, grad + (size_t)b * D, t);
}

// The coarse-stage loop: n_steps upper iterations (evaluate E, gradient,
// Adam, clamp) for B independent grasps, starting at step count t0 + 1.
// grad_mode 0: central differences (the definition), 1: analytic chain.
// x, mm, vv [B,D] are updated in place; E [B] receives E at the last
// evaluated pose.
void orc_run(void* h, void* o, double* x, double* mm, double* vv, int B, int n_steps, int t0, const double* params,
             const double* T, int s, int grad_mode, double fd_step, int threads, double* E) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const Params P = params_from(params);
  const int D = 6 + H.n;
  parallel_for(B, threads, [&](int b) {
    double* xb = x + (size_t)b * D;
    Vec g(D);
    for (int it = 0; it < n_steps; ++it) {
      Eval ev = evaluate(H, O, xb, P, T, s);
      if (E) E[b] = ev.E;
      if (grad_mode == 0) grad_fd(H, O, xb, P, T, s, fd_step, g.data());
      else grad_analytic(H, O, ev, P, T, s, g.data());
      adam_step(H, P, xb, mm + (size_t)b * D, vv + (size_t)b * D, g.data(), t0 + it + 1);
    }
  });
}

// Refinement energy, its gradient and the chosen samples at B poses.
//   pc [B,m,3] coarse-stage object points; E [B]; grad [B,D] (may be NULL);
//   kstar [B,m]; gap [B,m] (phi gap to the second-best sample, may be NULL).
void orc_refine_eval(void* h, void* o, const double* x, int B, const double* pc, double delta, double w_d,
                     double w_qp, int threads, double* E, double* grad, int32_t* kstar, double* gap) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const int D = 6 + H.n, m = H.m;
  parallel_for(B, threads, [&](int b) {
    Refine R = refine_eval(H, O, x + (size_t)b * D, pc + (size_t)b * m * 3, delta, w_d, w_qp,
                           grad ? grad + (size_t)b * D : nullptr);
    E[b] = R.E;
    for (int i = 0; i < m; ++i) {
      kstar[(size_t)b * m + i] = R.kstar[i];
      if (gap) gap[(size_t)b * m + i] = R.gap[i];
    }
  });
}

// Self-collision pairs of the hand (build_pairs): count, and [count,2] when out is given.
int orc_hand_pairs(void* h, int32_t* out) {
  const Hand& H = *static_cast<Hand*>(h);
  if (out)
    for (size_t k = 0; k < H.pairs.size(); ++k) {
      out[2 * k] = H.pairs[k].first;
      out[2 * k + 1] = H.pairs[k].second;
    }
  return (int)H.pairs.size();
}

// Signed fingertip distances d [B,m] and their spread cdc [B] (Sec. V-B).
void orc_contact_metrics(void* h, void* o, const double* x, int B, int threads, double* d, double* cdc) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const int D = 6 + H.n, m = H.m;
  parallel_for(B, threads, [&](int b) {
    Metrics R = contact_metrics(H, O, x + (size_t)b * D);
    for (int i = 0; i < m; ++i) d[(size_t)b * m + i] = R.d[i];
    cdc[b] = R.cdc;
  });
}

// n_steps refinement iterations (energy above, Adam + clamp) continuing at
// step count t0 + 1; x, mm, vv [B,D] in place; E [B] at the last evaluated pose.
void orc_refine_run(void* h, void* o, double* x, double* mm, double* vv, int B, const double* pc, int n_steps,
                    int t0, double delta, double w_qp, const double* params, int threads, double* E) {
  const Hand& H = *static_cast<Hand*>(h);
  const Object& O = *static_cast<Object*>(o);
  const Params P = params_from(params);
  const int D = 6 + H.n, m = H.m;
  parallel_for(B, threads, [&](int b) {
    double* xb = x + (size_t)b * D;
    Vec g(D);
    for (int it = 0; it < n_steps; ++it) {
      Refine R = refine_eval(H, O, xb, pc + (size_t)b * m * 3, delta, P.w_d, w_qp, g.data());
      if (E) E[b] = R.E;
      adam_step(H, P, xb, mm + (size_t)b * D, vv + (size_t)b * D, g.data(), t0 + it + 1);
    }
  });
}

}  // extern "C"
