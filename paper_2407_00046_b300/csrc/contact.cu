// Contact stencils on the GPU, FP64: unsigned point-triangle / edge-edge
// distances with region classification, the IPC clamped log barrier and the
// augmented-Lagrangian terms of Eq. (aug-lag), PSD projection of the 12x12
// stencil Hessian (Sec. 4.2.2), the fully-implicit friction of Sec. 4.1 on the
// same stencils (normal force, normal and closest-point weights lagged at the
// evaluation point), energies for the line search, the conservative step bound
// and the dual update of Algorithm 1.
//
// Region decisions (which closest-feature formula applies) and the distances
// used for set membership are computed with explicitly rounded operations
// (no fused multiply-add), so they round exactly like a plain left-to-right
// FP64 evaluation of the same formulas.
#include <cub/cub.cuh>

#include "scene.cuh"

namespace bal {

namespace {

enum { R_PP = 0, R_PE = 1, R_PT = 2, R_EE = 3 };
struct Region {
  int kind;
  int n[4];   // PP: (i, j); PE: (p, a, b); PT/EE: (0, 1, 2, 3)
};

// ---- explicitly rounded helpers ------------------------------------------------
__device__ inline d3 sub_rn(d3 a, d3 b) {
  return d3{__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)};
}
__device__ inline double dot_rn(d3 a, d3 b) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ inline d3 cross_rn(d3 a, d3 b) {
  return d3{__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)),
            __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}

// closest point on segment ab to p: squared distance, kind, which end (PP)
__device__ inline void seg_candidate(d3 p, d3 a, d3 b, double& d2, int& kind, int& end) {
  const d3 ab = sub_rn(b, a);
  const double L2 = dot_rn(ab, ab);
  const double u = L2 > 0.0 ? __ddiv_rn(dot_rn(sub_rn(p, a), ab), L2) : 0.0;
  if (u <= 0.0) {
    const d3 r = sub_rn(p, a);
    d2 = dot_rn(r, r);
    kind = R_PP;
    end = 0;
  } else if (u >= 1.0) {
    const d3 r = sub_rn(p, b);
    d2 = dot_rn(r, r);
    kind = R_PP;
    end = 1;
  } else {
    const d3 c = d3{__dadd_rn(a.x, __dmul_rn(u, ab.x)), __dadd_rn(a.y, __dmul_rn(u, ab.y)),
                    __dadd_rn(a.z, __dmul_rn(u, ab.z))};
    const d3 r = sub_rn(p, c);
    d2 = dot_rn(r, r);
    kind = R_PE;
    end = 0;
  }
}

__device__ inline Region make_seg_region(int kind, int end, int ip, int ia, int ib) {
  Region R;
  R.kind = kind;
  if (kind == R_PE) {
    R.n[0] = ip; R.n[1] = ia; R.n[2] = ib; R.n[3] = -1;
  } else {
    R.n[0] = ip; R.n[1] = end ? ib : ia; R.n[2] = -1; R.n[3] = -1;
  }
  return R;
}

__device__ Region classify_pt(const d3 X[4]) {
  const d3 e1 = sub_rn(X[2], X[1]), e2 = sub_rn(X[3], X[1]), r = sub_rn(X[0], X[1]);
  const double a11 = dot_rn(e1, e1), a12 = dot_rn(e1, e2), a22 = dot_rn(e2, e2);
  const double b1 = dot_rn(e1, r), b2 = dot_rn(e2, r);
  const double det = __dsub_rn(__dmul_rn(a11, a22), __dmul_rn(a12, a12));
  if (det > 0.0) {
    const double be1 = __ddiv_rn(__dsub_rn(__dmul_rn(a22, b1), __dmul_rn(a12, b2)), det);
    const double be2 = __ddiv_rn(__dsub_rn(__dmul_rn(a11, b2), __dmul_rn(a12, b1)), det);
    const double be0 = __dsub_rn(__dsub_rn(1.0, be1), be2);
    if (be0 > 0.0 && be1 > 0.0 && be2 > 0.0) {
      Region R;
      R.kind = R_PT;
      R.n[0] = 0; R.n[1] = 1; R.n[2] = 2; R.n[3] = 3;
      return R;
    }
  }
  const int ea[3] = {1, 2, 3}, eb[3] = {2, 3, 1};
  double best = 0.0;
  int bk = 0, bkind = 0, bend = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double d2;
    int kind, end;
    seg_candidate(X[0], X[ea[k]], X[eb[k]], d2, kind, end);
    if (k == 0 || d2 < best) {
      best = d2; bk = k; bkind = kind; bend = end;
    }
  }
  return make_seg_region(bkind, bend, 0, ea[bk], eb[bk]);
}

__device__ Region classify_ee(const d3 X[4]) {
  const d3 u = sub_rn(X[1], X[0]), v = sub_rn(X[3], X[2]), w = sub_rn(X[0], X[2]);
  const double A = dot_rn(u, u), B = dot_rn(u, v), C = dot_rn(v, v), D = dot_rn(u, w),
               Ev = dot_rn(v, w);
  const d3 n = cross_rn(u, v);
  const double den = dot_rn(n, n);
  if (den > __dmul_rn(__dmul_rn(1e-12, A), C)) {
    const double s = __ddiv_rn(__dsub_rn(__dmul_rn(B, Ev), __dmul_rn(C, D)), den);
    const double t = __ddiv_rn(__dsub_rn(__dmul_rn(A, Ev), __dmul_rn(B, D)), den);
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
      Region R;
      R.kind = R_EE;
      R.n[0] = 0; R.n[1] = 1; R.n[2] = 2; R.n[3] = 3;
      return R;
    }
  }
  const int ip[4] = {0, 1, 2, 3}, ia[4] = {2, 2, 0, 0}, ib[4] = {3, 3, 1, 1};
  double best = 0.0;
  int bk = 0, bkind = 0, bend = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double d2;
    int kind, end;
    seg_candidate(X[ip[k]], X[ia[k]], X[ib[k]], d2, kind, end);
    if (k == 0 || d2 < best) {
      best = d2; bk = k; bkind = kind; bend = end;
    }
  }
  return make_seg_region(bkind, bend, ip[bk], ia[bk], ib[bk]);
}

// distance of the region formula, explicitly rounded
__device__ double region_distance(const d3 X[4], const Region& R) {
  if (R.kind == R_PP) {
    const d3 r = sub_rn(X[R.n[0]], X[R.n[1]]);
    return __dsqrt_rn(dot_rn(r, r));
  }
  if (R.kind == R_PE) {
    const d3 e = sub_rn(X[R.n[2]], X[R.n[1]]);
    const d3 c = cross_rn(sub_rn(X[R.n[0]], X[R.n[1]]), e);
    return __dsqrt_rn(__ddiv_rn(dot_rn(c, c), dot_rn(e, e)));
  }
  if (R.kind == R_PT) {
    const d3 nrm = cross_rn(sub_rn(X[2], X[1]), sub_rn(X[3], X[1]));
    return __ddiv_rn(fabs(dot_rn(sub_rn(X[0], X[1]), nrm)), __dsqrt_rn(dot_rn(nrm, nrm)));
  }
  const d3 nrm = cross_rn(sub_rn(X[1], X[0]), sub_rn(X[3], X[2]));
  return __ddiv_rn(fabs(dot_rn(sub_rn(X[0], X[2]), nrm)), __dsqrt_rn(dot_rn(nrm, nrm)));
}

__device__ inline void pair_nodes(const Dev& S, uint64_t key, int v[4]) {
  const uint32_t a = key_a(key), b = key_b(key);
  if (key_kind(key) == 0) {
    v[0] = (int)a;
    v[1] = S.tris[3 * (int64_t)b];
    v[2] = S.tris[3 * (int64_t)b + 1];
    v[3] = S.tris[3 * (int64_t)b + 2];
  } else {
    v[0] = S.edges[2 * (int64_t)a];
    v[1] = S.edges[2 * (int64_t)a + 1];
    v[2] = S.edges[2 * (int64_t)b];
    v[3] = S.edges[2 * (int64_t)b + 1];
  }
}

__device__ inline double pair_distance(const Dev& S, const double* __restrict__ x, uint64_t key,
                                       int v[4], d3 X[4], Region& R) {
  pair_nodes(S, key, v);
#pragma unroll
  for (int a = 0; a < 4; ++a) X[a] = ld3(x, v[a]);
  R = key_kind(key) == 0 ? classify_pt(X) : classify_ee(X);
  return region_distance(X, R);
}

// ---- barrier (Sec. 3.3) ------------------------------------------------------------
__device__ inline double bar(double d, double c) {
  if (!(d > 0.0)) return INFINITY;
  if (d >= c) return 0.0;
  const double t = d - c;
  return -t * t * log(d / c);
}
__device__ inline double dbar(double d, double c) {
  if (!(d > 0.0) || d >= c) return 0.0;
  const double t = d - c;
  return -2.0 * t * log(d / c) - t * t / d;
}
__device__ inline double d2bar(double d, double c) {
  if (!(d > 0.0) || d >= c) return 0.0;
  const double t = d - c;
  return -2.0 * log(d / c) - 4.0 * t / d + t * t / (d * d);
}

// ---- edge-edge mollifier ------------------------------------------------------------
// The segment-segment distance is not C^1 where two edges turn parallel, so an
// exact Newton step cannot converge through such a configuration. Every
// edge-edge term is therefore scaled by m(c), c = |u x v|^2 with u, v the two
// edge vectors: m = (2 - c/eps) c/eps for c < eps = 1e-3 |u_rest|^2 |v_rest|^2,
// and 1 above (the mollifier of IPC, Li et al. 2020, whose barrier the paper
// uses; the paper itself is silent on parallel edges). m is C^1 at c = eps.
struct Mollifier {
  bool on;              // c < eps, i.e. m < 1
  double m, m1, m2;     // m, dm/dc, d2m/dc2
  d3 u, v;
};
__device__ inline Mollifier ee_mollifier(const Dev& S, uint64_t key, const d3 X[4]) {
  Mollifier M;
  M.on = false;
  M.m = 1.0;
  M.m1 = M.m2 = 0.0;
  M.u = X[1] - X[0];
  M.v = X[3] - X[2];
  if (key_kind(key) == 0) return M;
  const double eps = 1e-3 * S.edge_l2[key_a(key)] * S.edge_l2[key_b(key)];
  const d3 n = cross(M.u, M.v);
  const double c = dot(n, n);
  if (!(c < eps)) return M;
  const double r = c / eps;
  M.on = true;
  M.m = (2.0 - r) * r;
  M.m1 = (2.0 - 2.0 * r) / eps;
  M.m2 = -2.0 / (eps * eps);
  return M;
}
// grad c on the 12 stencil DOFs: c = |u|^2 |v|^2 - (u.v)^2 with u = X1 - X0,
// v = X3 - X2, so dc/du = 2|v|^2 u - 2(u.v) v and dc/dv = 2|u|^2 v - 2(u.v) u
__device__ inline void mollifier_grad_c(const Mollifier& M, double gc[12]) {
  const double uu = dot(M.u, M.u), vv = dot(M.v, M.v), uv = dot(M.u, M.v);
  const d3 gu = (2.0 * vv) * M.u - (2.0 * uv) * M.v;
  const d3 gv = (2.0 * uu) * M.v - (2.0 * uv) * M.u;
  const d3 g[4] = {-1.0 * gu, gu, -1.0 * gv, gv};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    gc[3 * k] = g[k].x;
    gc[3 * k + 1] = g[k].y;
    gc[3 * k + 2] = g[k].z;
  }
}
// entry (r, c) of the Hessian of c on the 12 DOFs: with e_uu = 2|v|^2 I - 2 v v^T,
// e_vv = 2|u|^2 I - 2 u u^T, e_uv = 4 u v^T - 2(u.v) I - 2 v u^T, e_vu = e_uv^T,
// signed by the node's sign in u or v (X0, X2: -1; X1, X3: +1)
__device__ inline double mollifier_hess_c(const Mollifier& M, int r, int c, double uu, double vv,
                                          double uv) {
  const int a = r / 3, i = r % 3, b = c / 3, j = c % 3;
  const double sgn = ((a & 1) ? 1.0 : -1.0) * ((b & 1) ? 1.0 : -1.0);
  const double u[3] = {M.u.x, M.u.y, M.u.z}, v[3] = {M.v.x, M.v.y, M.v.z};
  const double dij = i == j ? 1.0 : 0.0;
  double e;
  if (a < 2 && b < 2) e = 2.0 * vv * dij - 2.0 * v[i] * v[j];
  else if (a >= 2 && b >= 2) e = 2.0 * uu * dij - 2.0 * u[i] * u[j];
  else if (a < 2) e = 4.0 * u[i] * v[j] - 2.0 * uv * dij - 2.0 * v[i] * u[j];
  else e = 4.0 * u[j] * v[i] - 2.0 * uv * dij - 2.0 * v[j] * u[i];
  return sgn * e;
}

// ---- derivatives of d^2 (hand-derived, per region) ----------------------------------
// Variables are differences of stencil nodes: var_k = sum_n C[k][n] X[n] with C in
// {-1,0,1}. f = d^2(vars); fk[k] = df/dvar_k; Fkl[k][l] = d2f/dvar_k dvar_l (3x3).
struct VarSpace {
  int nvar;
  int C[3][4];
  d3 fk[3];
  double Fkl[3][3][3][3];
  double f;
};

__device__ inline void outer_acc(double M[3][3], double s, d3 a, d3 b) {
  const double av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] += s * av[i] * bv[j];
}
__device__ inline void skew_acc(double M[3][3], double s, d3 a) {   // M += s [a]x
  M[0][1] -= s * a.z; M[0][2] += s * a.y;
  M[1][0] += s * a.z; M[1][2] -= s * a.x;
  M[2][0] -= s * a.y; M[2][1] += s * a.x;
}
__device__ inline void eye_acc(double M[3][3], double s) {
  M[0][0] += s; M[1][1] += s; M[2][2] += s;
}

__device__ void d2_derivs(const d3 X[4], const Region& R, VarSpace& V) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int n = 0; n < 4; ++n) V.C[k][n] = 0;
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V.Fkl[k][l][i][j] = 0.0;
  }
  if (R.kind == R_PP) {
    V.nvar = 1;
    V.C[0][R.n[0]] = 1;
    V.C[0][R.n[1]] = -1;
    const d3 r = X[R.n[0]] - X[R.n[1]];
    V.f = dot(r, r);
    V.fk[0] = 2.0 * r;
    eye_acc(V.Fkl[0][0], 2.0);
    return;
  }
  if (R.kind == R_PE) {
    V.nvar = 2;
    V.C[0][R.n[0]] = 1; V.C[0][R.n[1]] = -1;   // u = p - a
    V.C[1][R.n[2]] = 1; V.C[1][R.n[1]] = -1;   // e = b - a
    const d3 u = X[R.n[0]] - X[R.n[1]], e = X[R.n[2]] - X[R.n[1]];
    const double k = dot(u, e), L = dot(e, e), iL = 1.0 / L;
    V.f = dot(u, u) - k * k * iL;
    V.fk[0] = 2.0 * u - (2.0 * k * iL) * e;
    V.fk[1] = (2.0 * k * k * iL * iL) * e - (2.0 * k * iL) * u;
    eye_acc(V.Fkl[0][0], 2.0);
    outer_acc(V.Fkl[0][0], -2.0 * iL, e, e);
    outer_acc(V.Fkl[0][1], -2.0 * iL, e, u);
    eye_acc(V.Fkl[0][1], -2.0 * k * iL);
    outer_acc(V.Fkl[0][1], 4.0 * k * iL * iL, e, e);
    outer_acc(V.Fkl[1][1], -2.0 * iL, u, u);
    outer_acc(V.Fkl[1][1], 4.0 * k * iL * iL, u, e);
    outer_acc(V.Fkl[1][1], 4.0 * k * iL * iL, e, u);
    eye_acc(V.Fkl[1][1], 2.0 * k * k * iL * iL);
    outer_acc(V.Fkl[1][1], -8.0 * k * k * iL * iL * iL, e, e);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) V.Fkl[1][0][i][j] = V.Fkl[0][1][j][i];
    return;
  }
  // plane distance: f = u^2 / w, u = r . (a x b), w = |a x b|^2
  V.nvar = 3;
  d3 r, a, b;
  if (R.kind == R_PT) {   // r = X0 - X1, a = X2 - X1, b = X3 - X1
    V.C[0][0] = 1; V.C[0][1] = -1;
    V.C[1][2] = 1; V.C[1][1] = -1;
    V.C[2][3] = 1; V.C[2][1] = -1;
    r = X[0] - X[1]; a = X[2] - X[1]; b = X[3] - X[1];
  } else {                // r = X0 - X2, a = X1 - X0, b = X3 - X2
    V.C[0][0] = 1; V.C[0][2] = -1;
    V.C[1][1] = 1; V.C[1][0] = -1;
    V.C[2][3] = 1; V.C[2][2] = -1;
    r = X[0] - X[2]; a = X[1] - X[0]; b = X[3] - X[2];
  }
  const d3 n = cross(a, b);
  const double u = dot(r, n), w = dot(n, n), iw = 1.0 / w;
  const d3 gu[3] = {n, cross(b, r), cross(r, a)};
  const d3 gw[3] = {d3{0, 0, 0}, 2.0 * cross(b, n), 2.0 * cross(n, a)};
  V.f = u * u * iw;
  const double c_u = 2.0 * u * iw, c_w = -u * u * iw * iw;
#pragma unroll
  for (int k = 0; k < 3; ++k) V.fk[k] = c_u * gu[k] + c_w * gw[k];
  const double al = 2.0 * iw, be = -2.0 * u * iw * iw, ga = 2.0 * u * u * iw * iw * iw;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      outer_acc(V.Fkl[k][l], al, gu[k], gu[l]);
      outer_acc(V.Fkl[k][l], be, gu[k], gw[l]);
      outer_acc(V.Fkl[k][l], be, gw[k], gu[l]);
      outer_acc(V.Fkl[k][l], ga, gw[k], gw[l]);
    }
  // + (2u/w) Hess u : U_ra = -[b]x, U_rb = [a]x, U_ab = -[r]x (and transposes)
  const double su = 2.0 * u * iw;
  skew_acc(V.Fkl[0][1], -su, b);
  skew_acc(V.Fkl[1][0], su, b);
  skew_acc(V.Fkl[0][2], su, a);
  skew_acc(V.Fkl[2][0], -su, a);
  skew_acc(V.Fkl[1][2], -su, r);
  skew_acc(V.Fkl[2][1], su, r);
  // - (u^2/w^2) Hess w : W_aa = 2(|b|^2 I - b b^T), W_bb = 2(|a|^2 I - a a^T),
  //                      W_ab = 2(2 a b^T - (a.b) I - b a^T)
  const double sw = -u * u * iw * iw;
  eye_acc(V.Fkl[1][1], 2.0 * sw * dot(b, b));
  outer_acc(V.Fkl[1][1], -2.0 * sw, b, b);
  eye_acc(V.Fkl[2][2], 2.0 * sw * dot(a, a));
  outer_acc(V.Fkl[2][2], -2.0 * sw, a, a);
  outer_acc(V.Fkl[1][2], 4.0 * sw, a, b);
  eye_acc(V.Fkl[1][2], -2.0 * sw * dot(a, b));
  outer_acc(V.Fkl[1][2], -2.0 * sw, b, a);
  outer_acc(V.Fkl[2][1], 4.0 * sw, b, a);
  eye_acc(V.Fkl[2][1], -2.0 * sw * dot(a, b));
  outer_acc(V.Fkl[2][1], -2.0 * sw, a, b);
}

// ---- 12x12 symmetric eigen-decomposition by cyclic Jacobi ------------------------
// A (row-major 144) is overwritten (diagonal = eigenvalues); Q gets the eigenvectors
// in its columns. Bounded sweep count; off-diagonal mass checked every sweep.
__device__ void jacobi12(double* A, double* Q) {
  for (int i = 0; i < 144; ++i) Q[i] = (i % 13 == 0) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < 144; ++i) fro += A[i] * A[i];
  if (fro == 0.0) return;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 12; ++p)
      for (int q = p + 1; q < 12; ++q) off += A[12 * p + q] * A[12 * p + q];
    if (off <= 1e-32 * fro) break;
    for (int p = 0; p < 11; ++p) {
      for (int q = p + 1; q < 12; ++q) {
        const double apq = A[12 * p + q];
        if (fabs(apq) <= 1e-300) continue;
        const double app = A[13 * p], aqq = A[13 * q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < 12; ++r) {
          if (r == p || r == q) continue;
          const double arp = A[12 * r + p], arq = A[12 * r + q];
          const double nrp = c * arp - s * arq, nrq = s * arp + c * arq;
          A[12 * r + p] = A[12 * p + r] = nrp;
          A[12 * r + q] = A[12 * q + r] = nrq;
        }
        A[13 * p] = app - t * apq;
        A[13 * q] = aqq + t * apq;
        A[12 * p + q] = A[12 * q + p] = 0.0;
        for (int r = 0; r < 12; ++r) {
          const double vrp = Q[12 * r + p], vrq = Q[12 * r + q];
          Q[12 * r + p] = c * vrp - s * vrq;
          Q[12 * r + q] = s * vrp + c * vrq;
        }
      }
    }
  }
}

// ---- friction (Sec. 4.1) ------------------------------------------------------------
// Signed weights of the two closest points of a stencil in region R, so that
// sum_k beta_k X_k runs from the closest point of the second primitive to that
// of the first (first primitive's weights >= 0).
__device__ void closest_weights(const d3 X[4], const Region& R, double beta[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) beta[k] = 0.0;
  if (R.kind == R_PP) {
    beta[R.n[0]] = 1.0;
    beta[R.n[1]] = -1.0;
  } else if (R.kind == R_PE) {
    const d3 e = X[R.n[2]] - X[R.n[1]];
    const double t = dot(X[R.n[0]] - X[R.n[1]], e) / dot(e, e);
    beta[R.n[0]] = 1.0;
    beta[R.n[1]] = -(1.0 - t);
    beta[R.n[2]] = -t;
  } else if (R.kind == R_PT) {
    // projection of X0 on the triangle's plane: 2x2 normal equations
    const d3 e1 = X[2] - X[1], e2 = X[3] - X[1], r = X[0] - X[1];
    const double a11 = dot(e1, e1), a12 = dot(e1, e2), a22 = dot(e2, e2);
    const double r1 = dot(e1, r), r2 = dot(e2, r);
    const double det = a11 * a22 - a12 * a12;
    const double b1 = (a22 * r1 - a12 * r2) / det, b2 = (a11 * r2 - a12 * r1) / det;
    beta[0] = 1.0;
    beta[1] = -(1.0 - b1 - b2);
    beta[2] = -b1;
    beta[3] = -b2;
  } else {
    // line-line closest parameters s (edge a), t (edge b)
    const d3 u = X[1] - X[0], v = X[3] - X[2], w = X[0] - X[2];
    const double A = dot(u, u), B = dot(u, v), C = dot(v, v), D = dot(u, w), E = dot(v, w);
    const double den = A * C - B * B;
    const double s = (B * E - C * D) / den, t = (A * E - B * D) / den;
    beta[0] = 1.0 - s;
    beta[1] = s;
    beta[2] = -(1.0 - t);
    beta[3] = -t;
  }
  if (beta[0] + beta[1] < 0.0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) beta[k] = -beta[k];
  }
}

// Tangent slip w = P sum_k beta_k (X_k - X^t_k) with P = I - nh nh^T.
__device__ inline d3 tangent_slip(const double beta[4], const d3 X[4], const d3 Xt[4], d3 nh) {
  d3 u = d3{0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) u = u + beta[k] * (X[k] - Xt[k]);
  return u - dot(u, nh) * nh;
}

// Mollified slip magnitude f(y) (Sec. 4.1): the printed cubic below eps h,
// continued linearly (C^2) beyond.
__device__ inline double fric_f(double y, double eh) {
  return y < eh ? y * y / eh - y * y * y / (3.0 * eh * eh) : y - eh / 3.0;
}

// lagged friction set read by the line-search energy
struct FricLag {
  const uint64_t* keys;
  const double *beta, *nrm, *lam, *xt;
  int64_t n;
  double chi, eps_h;
};

struct ContactArgs {
  const uint64_t* keys;
  const uint8_t* flags;
  const double* mu;
  const double* s;
  int64_t n;
  double sigma;
  double* grad;
  int hess;
  uint64_t* emit_keys;   // [n][6]
  double* emit_vals;     // [n][6][9]
  int project;           // 0: emit the unprojected stencil Hessian (adjoint)
  // friction (Sec. 4.1), lagged at x: off when fric == 0
  int fric;
  double chi, eps_h;     // friction coefficient, eps_v h
  const double* xt;      // start of the time step
  double* fr_beta;       // [n][4] lagged weights (written)
  double* fr_n;          // [n][3] lagged unit normals (written)
  double* fr_lam;        // [n] lagged normal forces (written)
};

__global__ void __launch_bounds__(128) k_contact_terms(Dev S, const double* __restrict__ x,
                                                       ContactArgs A) {
  double H[144], Q[144];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = A.keys[i];
    int v[4];
    d3 X[4];
    Region R;
    pair_distance(S, x, key, v, X, R);
    VarSpace V;
    d2_derivs(X, R, V);
    const double d = sqrt(V.f);
    const uint8_t fl = A.flags[i];
    const double inA = (fl & PF_A) ? 1.0 : 0.0, inAp = (fl & PF_AP) ? 1.0 : 0.0;
    const double c2 = S.dhat + A.s[i];
    const double p1 = inA * A.sigma * dbar(d, S.dhat) + inAp * (-A.mu[i] + A.sigma * dbar(d, c2));
    const double p2 = inA * A.sigma * d2bar(d, S.dhat) + inAp * A.sigma * d2bar(d, c2);
    // edge-edge mollifier: phi_EE = m phi, grad = m phi' grad d + phi m' grad c
    const Mollifier M = ee_mollifier(S, key, X);
    double e0 = 0.0, gc[12];
    if (M.on) {
      e0 = inA * A.sigma * bar(d, S.dhat) + inAp * (A.mu[i] * (c2 - d) + A.sigma * bar(d, c2));
      mollifier_grad_c(M, gc);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) gc[k] = 0.0;
    }
    // g2 = grad(d^2) on the 12 stencil DOFs
    double g2[12];
#pragma unroll
    for (int nd = 0; nd < 4; ++nd) {
      d3 acc = d3{0, 0, 0};
      for (int k = 0; k < V.nvar; ++k)
        if (V.C[k][nd] != 0) acc = acc + (double)V.C[k][nd] * V.fk[k];
      g2[3 * nd] = acc.x; g2[3 * nd + 1] = acc.y; g2[3 * nd + 2] = acc.z;
    }
    const double cg = M.m * p1 / (2.0 * d), cm = e0 * M.m1;
    // friction: normal force lambda = -m phi'(d), normal and weights at x; the
    // slip w against x^t; D = chi lambda f(|w|), grad = chi lambda a beta_k w,
    // Hess block (k, l) = chi lambda beta_k beta_l (a P + c w w^T)
    double beta[4] = {0, 0, 0, 0}, fk = 0.0, fa = 0.0, fcy = 0.0;
    d3 nh = d3{0, 0, 0}, w = d3{0, 0, 0};
    if (A.fric) {
      closest_weights(X, R, beta);
      d3 nv = d3{0, 0, 0}, Xt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        nv = nv + beta[k] * X[k];
        Xt[k] = ld3(A.xt, v[k]);
      }
      nh = (1.0 / sqrt(dot(nv, nv))) * nv;
      w = tangent_slip(beta, X, Xt, nh);
      const double lam = -M.m * p1;
      fk = A.chi * lam;
      const double y = sqrt(dot(w, w)), eh = A.eps_h;
      if (y < eh) {
        fa = 2.0 / eh - y / (eh * eh);
        fcy = y > 0.0 ? -1.0 / (eh * eh * y) : 0.0;
      } else {
        fa = 1.0 / y;
        fcy = -1.0 / (y * y * y);
      }
      if (A.fr_lam) {
#pragma unroll
        for (int k = 0; k < 4; ++k) A.fr_beta[4 * i + k] = beta[k];
        A.fr_n[3 * i] = nh.x;
        A.fr_n[3 * i + 1] = nh.y;
        A.fr_n[3 * i + 2] = nh.z;
        A.fr_lam[i] = lam;
      }
    }
    bool pin[4];
#pragma unroll
    for (int nd = 0; nd < 4; ++nd) {
      pin[nd] = S.pinned[v[nd]] != 0;
      if (!pin[nd] && A.grad) {
        const double cf = fk * fa * beta[nd];
        atomic_add3(A.grad, v[nd], d3{cg * g2[3 * nd] + cm * gc[3 * nd] + cf * w.x,
                                      cg * g2[3 * nd + 1] + cm * gc[3 * nd + 1] + cf * w.y,
                                      cg * g2[3 * nd + 2] + cm * gc[3 * nd + 2] + cf * w.z});
      }
    }
    if (!A.hess) continue;
    // H = c1 g2 g2^T + c2 Hess(d^2)
    const double c1 = (p2 - p1 / d) / (4.0 * d * d), cc2 = p1 / (2.0 * d);
    for (int nd = 0; nd < 4; ++nd)
      for (int md = 0; md < 4; ++md)
        for (int ii = 0; ii < 3; ++ii)
          for (int jj = 0; jj < 3; ++jj) {
            double h2 = 0.0;
            for (int k = 0; k < V.nvar; ++k) {
              const int ck = V.C[k][nd];
              if (!ck) continue;
              for (int l = 0; l < V.nvar; ++l) {
                const int cl = V.C[l][md];
                if (cl) h2 += (double)(ck * cl) * V.Fkl[k][l][ii][jj];
              }
            }
            const int r = 3 * nd + ii, c = 3 * md + jj;
            H[12 * r + c] = c1 * g2[r] * g2[c] + cc2 * h2;
          }
    if (M.on) {
      // m (phi'' grad d grad d^T + phi' Hess d) + phi' m' (grad d grad c^T + grad c grad d^T)
      // + phi (m'' grad c grad c^T + m' Hess c)
      const double uu = dot(M.u, M.u), vv = dot(M.v, M.v), uv = dot(M.u, M.v);
      const double cx = p1 * M.m1 / (2.0 * d), cgg = e0 * M.m2, chc = e0 * M.m1;
      for (int r = 0; r < 12; ++r)
        for (int c = 0; c < 12; ++c)
          H[12 * r + c] = M.m * H[12 * r + c] + cx * (g2[r] * gc[c] + gc[r] * g2[c]) +
                          cgg * gc[r] * gc[c] + chc * mollifier_hess_c(M, r, c, uu, vv, uv);
    }
    // symmetrise, project to PSD
    for (int r = 0; r < 12; ++r)
      for (int c = r + 1; c < 12; ++c) {
        const double m = 0.5 * (H[12 * r + c] + H[12 * c + r]);
        H[12 * r + c] = H[12 * c + r] = m;
      }
    double tr = 0.0;
    if (A.project) {
      jacobi12(H, Q);
      double lam[12];
      for (int k = 0; k < 12; ++k) {
        lam[k] = H[13 * k] > 0.0 ? H[13 * k] : 0.0;
        tr += lam[k];
      }
      for (int r = 0; r < 12; ++r)
        for (int c = r; c < 12; ++c) {
          double acc = 0.0;
          for (int k = 0; k < 12; ++k) acc += Q[12 * r + k] * lam[k] * Q[12 * c + k];
          H[12 * r + c] = H[12 * c + r] = acc;
        }
    } else {
      for (int k = 0; k < 12; ++k) tr += H[13 * k];
    }
    if (A.fric && fk > 0.0) {   // friction stencil: PSD by construction, added after the projection
      const double wv[3] = {w.x, w.y, w.z}, nvv[3] = {nh.x, nh.y, nh.z};
      double M[3][3];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
          M[ii][jj] = fa * ((ii == jj ? 1.0 : 0.0) - nvv[ii] * nvv[jj]) + fcy * wv[ii] * wv[jj];
      double b2 = 0.0;
      for (int nd = 0; nd < 4; ++nd) {
        b2 += beta[nd] * beta[nd];
        for (int md = 0; md < 4; ++md) {
          const double s = fk * beta[nd] * beta[md];
          for (int ii = 0; ii < 3; ++ii)
            for (int jj = 0; jj < 3; ++jj) H[12 * (3 * nd + ii) + 3 * md + jj] += s * M[ii][jj];
        }
      }
      tr += fk * b2 * (M[0][0] + M[1][1] + M[2][2]);
    }
    tr *= (1.0 / 12.0);
#pragma unroll
    for (int nd = 0; nd < 4; ++nd) {
      atomicAdd(S.Lambda + 3 * v[nd], tr);
      atomicAdd(S.Lambda + 3 * v[nd] + 1, tr);
      atomicAdd(S.Lambda + 3 * v[nd] + 2, tr);
      if (!pin[nd]) {
        double* Dd = S.D + 9 * (int64_t)v[nd];
        for (int ii = 0; ii < 3; ++ii)
          for (int jj = 0; jj < 3; ++jj) atomicAdd(Dd + 3 * ii + jj, H[12 * (3 * nd + ii) + 3 * nd + jj]);
      }
    }
    // off-diagonal lower blocks -> (key = row << 32 | col, value) for the segmented reduction
    const int pa[6] = {1, 2, 3, 2, 3, 3};
    const int pb[6] = {0, 0, 0, 1, 1, 2};
    for (int k = 0; k < 6; ++k) {
      const int a = pa[k], b = pb[k];
      uint64_t* ek = A.emit_keys + 6 * i + k;
      double* ev = A.emit_vals + 9 * (6 * i + k);
      if (pin[a] || pin[b]) {
        *ek = ~0ull;
        continue;
      }
      const bool a_row = v[a] > v[b];
      const int rn = a_row ? a : b, cn = a_row ? b : a;
      *ek = ((uint64_t)(uint32_t)v[rn] << 32) | (uint32_t)v[cn];
      for (int ii = 0; ii < 3; ++ii)
        for (int jj = 0; jj < 3; ++jj) ev[3 * ii + jj] = H[12 * (3 * rn + ii) + 3 * cn + jj];
    }
  }
}

__global__ void k_pair_distance(Dev S, const double* __restrict__ x, const uint64_t* __restrict__ keys,
                                int64_t n, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    Region R;
    d[i] = pair_distance(S, x, keys[i], v, X, R);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_contact_energy(Dev S, const double* __restrict__ x,
                                                       const uint64_t* __restrict__ cand, int64_t nc,
                                                       const uint64_t* __restrict__ apk,
                                                       const double* __restrict__ apmu,
                                                       const double* __restrict__ aps, int64_t nap,
                                                       double sigma, FricLag F, double* partials, int nblk) {
  double e = 0.0, cnt = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < nc; i += (int64_t)gridDim.x * NT) {
    int v[4];
    d3 X[4];
    Region R;
    const double d = pair_distance(S, x, cand[i], v, X, R);
    if (d < S.dhat) {
      e += ee_mollifier(S, cand[i], X).m * sigma * bar(d, S.dhat);
      cnt += 1.0;
    }
  }
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < nap; i += (int64_t)gridDim.x * NT) {
    int v[4];
    d3 X[4];
    Region R;
    const double d = pair_distance(S, x, apk[i], v, X, R);
    const double c2 = S.dhat + aps[i];
    e += ee_mollifier(S, apk[i], X).m * (apmu[i] * (c2 - d) + sigma * bar(d, c2));
  }
  // friction with the lagged weights, normals and forces
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < F.n; i += (int64_t)gridDim.x * NT) {
    int v[4];
    pair_nodes(S, F.keys[i], v);
    d3 X[4], Xt[4];
    double beta[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      X[k] = ld3(x, v[k]);
      Xt[k] = ld3(F.xt, v[k]);
      beta[k] = F.beta[4 * i + k];
    }
    const d3 w = tangent_slip(beta, X, Xt, ld3(F.nrm, (int)i));
    e += F.chi * F.lam[i] * fric_f(sqrt(dot(w, w)), F.eps_h);
  }
  e = block_sum<double, NT>(e);
  cnt = block_sum<double, NT>(cnt);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = e;
    partials[nblk + blockIdx.x] = cnt;
  }
}

// Step bound by conservative advancement: along x + t p a pair's distance can
// shrink by at most Delta per unit t (Delta = max |p_a - p_b| over a node of
// each primitive), so from t it is safe to advance by (d(t) - (1 - eta) d0) /
// Delta. Iterate to the time at which the distance would reach (1 - eta) d0,
// or to t = 1, at most max_iter times; the block minimum of t goes to partials.
template <int NT>
__global__ void __launch_bounds__(NT) k_step_bound(Dev S, const double* __restrict__ x,
                                                   const double* __restrict__ dir,
                                                   const uint64_t* __restrict__ cand, int64_t nc,
                                                   double eta, int max_iter, double* partials) {
  double amin = 1.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < nc; i += (int64_t)gridDim.x * NT) {
    int v[4];
    d3 X[4];
    Region R;
    const uint64_t key = cand[i];
    const double d0 = pair_distance(S, x, key, v, X, R);
    d3 P[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) P[a] = ld3(dir, v[a]);
    const int na = key_kind(key) == 0 ? 1 : 2;
    double Dl = 0.0;
    for (int a = 0; a < na; ++a)
      for (int b = na; b < 4; ++b) {
        const d3 w = P[a] - P[b];
        Dl = fmax(Dl, sqrt(dot(w, w)));
      }
    if (!(eta * d0 < Dl)) continue;
    const double goal = (1.0 - eta) * d0;
    double t = 0.0;
    for (int it = 0; it < max_iter; ++it) {
      d3 Xt[4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        Xt[a] = d3{__dadd_rn(X[a].x, __dmul_rn(t, P[a].x)), __dadd_rn(X[a].y, __dmul_rn(t, P[a].y)),
                   __dadd_rn(X[a].z, __dmul_rn(t, P[a].z))};
      const Region Rt = key_kind(key) == 0 ? classify_pt(Xt) : classify_ee(Xt);
      const double dk = region_distance(Xt, Rt);
      const double step = (dk - goal) / Dl;
      if (step <= 1e-6 * fmax(t, 1e-3)) break;      // at the offset time of impact
      const double nt = t + step;
      if (nt >= 1.0) {
        t = 1.0;
        break;
      }
      t = nt;
    }
    amin = fmin(amin, t);
  }
  amin = block_min<double, NT>(amin, 1.0);
  if (threadIdx.x == 0) partials[blockIdx.x] = amin;
}

// ---- cubic CCD with a conservative time of impact (Sec. 5.3, narrow phase) ----
// x(t) = x + t p; the stencil's nodes are coplanar where the triple product
// f(t) = ((t1 - t0) x (t2 - t0)) . (p - t0) (PT) or ((a1 - a0) x (b1 - b0)) .
// (b0 - a0) (EE) vanishes, a cubic in t. Every step is written with the
// round-to-nearest intrinsics so that no product is contracted into an FMA.
struct Cubic {
  double c0, c1, c2, c3;
};
__device__ inline d3 add_rn(d3 a, d3 b) { return d3{__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)}; }
__device__ Cubic coplanarity_cubic(const d3 X[4], const d3 P[4], bool ee) {
  d3 u0, u1, w0, w1, v0, v1;
  if (ee) {
    u0 = sub_rn(X[1], X[0]); u1 = sub_rn(P[1], P[0]);
    w0 = sub_rn(X[3], X[2]); w1 = sub_rn(P[3], P[2]);
    v0 = sub_rn(X[2], X[0]); v1 = sub_rn(P[2], P[0]);
  } else {
    u0 = sub_rn(X[2], X[1]); u1 = sub_rn(P[2], P[1]);
    w0 = sub_rn(X[3], X[1]); w1 = sub_rn(P[3], P[1]);
    v0 = sub_rn(X[0], X[1]); v1 = sub_rn(P[0], P[1]);
  }
  const d3 n0 = cross_rn(u0, w0), n1 = add_rn(cross_rn(u0, w1), cross_rn(u1, w0)), n2 = cross_rn(u1, w1);
  return Cubic{dot_rn(n0, v0), __dadd_rn(dot_rn(n0, v1), dot_rn(n1, v0)), __dadd_rn(dot_rn(n1, v1), dot_rn(n2, v0)),
               dot_rn(n2, v1)};
}
__device__ inline double cubic_at(const Cubic& c, double t) {
  return __dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(c.c3, t), c.c2), t), c.c1), t), c.c0);
}
__device__ inline double cubic_slope(const Cubic& c, double t) {
  return __dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(__dmul_rn(3.0, c.c3), t), __dmul_rn(2.0, c.c2)), t), c.c1);
}
// real roots of a t^2 + b t + c, ascending; returns the count (0..2)
__device__ int quadratic_roots(double a, double b, double c, double r[2]) {
  if (a == 0.0) {
    if (b == 0.0) return 0;
    r[0] = __ddiv_rn(-c, b);
    return 1;
  }
  const double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(__dmul_rn(4.0, a), c));
  if (disc < 0.0) return 0;
  const double sq = __dsqrt_rn(disc);
  const double q = __dmul_rn(-0.5, __dadd_rn(b, copysign(sq, b)));
  if (q == 0.0) {
    r[0] = __ddiv_rn(q, a);
    return 1;
  }
  const double x0 = __ddiv_rn(q, a), x1 = __ddiv_rn(c, q);
  r[0] = fmin(x0, x1);
  r[1] = fmax(x0, x1);
  return 2;
}
// root in [lo, hi], sign(f(lo)) = sign(flo) != sign(f(hi)): Newton steps kept
// inside the bracket, bisection otherwise
__device__ double newton_bisect(const Cubic& c, double lo, double hi, double flo) {
  double t = __dmul_rn(0.5, __dadd_rn(lo, hi));
  for (int it = 0; it < 200; ++it) {
    const double ft = cubic_at(c, t);
    if (ft == 0.0) return t;
    if ((ft > 0) == (flo > 0)) lo = t;
    else hi = t;
    const double d = cubic_slope(c, t);
    double tn = d != 0.0 ? __dsub_rn(t, __ddiv_rn(ft, d)) : __dmul_rn(0.5, __dadd_rn(lo, hi));
    if (!(lo < tn && tn < hi)) tn = __dmul_rn(0.5, __dadd_rn(lo, hi));
    if (fabs(__dsub_rn(tn, t)) <= __dmul_rn(1e-15, fmax(1.0, fabs(t))) || __dsub_rn(hi, lo) <= 1e-16) return tn;
    t = tn;
  }
  return t;
}
// coplanar times in [lo, hi], ascending (first root, then the deflated quadratic)
__device__ int coplanar_times(const Cubic& c, double lo, double hi, double out[3]) {
  double crit[2];
  const int nc = quadratic_roots(__dmul_rn(3.0, c.c3), __dmul_rn(2.0, c.c2), c.c1, crit);
  double knots[4];
  int nk = 0;
  knots[nk++] = lo;
  for (int k = 0; k < nc; ++k)
    if (lo < crit[k] && crit[k] < hi) knots[nk++] = crit[k];
  knots[nk++] = hi;
  double t0 = 0.0;
  bool found = false;
  for (int k = 0; k + 1 < nk && !found; ++k) {
    const double fa = cubic_at(c, knots[k]), fb = cubic_at(c, knots[k + 1]);
    if (fa == 0.0) {
      t0 = knots[k];
      found = true;
    } else if ((fa > 0) != (fb > 0) || fb == 0.0) {
      t0 = fb == 0.0 ? knots[k + 1] : newton_bisect(c, knots[k], knots[k + 1], fa);
      found = true;
    }
  }
  if (!found) return 0;
  int n = 0;
  out[n++] = t0;
  const double A = c.c3, B = __dadd_rn(c.c2, __dmul_rn(A, t0)), C = __dadd_rn(c.c1, __dmul_rn(B, t0));
  double r[2];
  const int nr = quadratic_roots(A, B, C, r);
  for (int k = 0; k < nr; ++k)
    if (t0 < r[k] && r[k] <= hi) out[n++] = r[k];
  return n;
}

// Conservative time of impact of each candidate along x + t dir times the
// line-search margin (1 when the pair does not activate); block minima into
// partials.
template <int NT>
__global__ void __launch_bounds__(NT) k_ccd_toi(Dev S, const double* __restrict__ x,
                                                const double* __restrict__ dir,
                                                const uint64_t* __restrict__ cand, int64_t nc,
                                                double eta_margin, double* partials) {
  const double eps = 1e-12;
  double amin = 1.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < nc; i += (int64_t)gridDim.x * NT) {
    int v[4];
    d3 X[4];
    Region R;
    const uint64_t key = cand[i];
    const double d0 = pair_distance(S, x, key, v, X, R);
    d3 P[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) P[a] = ld3(dir, v[a]);
    const bool ee = key_kind(key) != 0;
    const Cubic c = coplanarity_cubic(X, P, ee);
    // activation threshold: dhat + eps from outside the barrier's support, a
    // touch (eps) for a pair already inside it
    const double thr = d0 >= S.dhat ? __dadd_rn(eps, S.dhat) : eps;
    double ex = 0.0, ep = 0.0;
    for (int a = 0; a < 4; ++a) {
      ex = fmax(ex, fmax(fabs(__dsub_rn(X[a].x, X[0].x)), fmax(fabs(__dsub_rn(X[a].y, X[0].y)), fabs(__dsub_rn(X[a].z, X[0].z)))));
      ep = fmax(ep, fmax(fabs(__dsub_rn(P[a].x, P[0].x)), fmax(fabs(__dsub_rn(P[a].y, P[0].y)), fabs(__dsub_rn(P[a].z, P[0].z)))));
    }
    const double L = __dadd_rn(ex, ep);
    const double cmax = fmax(fmax(fabs(c.c0), fabs(c.c1)), fmax(fabs(c.c2), fabs(c.c3)));
    if (L == 0.0 || cmax <= __dmul_rn(1e-14, __dmul_rn(__dmul_rn(L, L), L))) continue;
    double ts[3];
    const int nt = coplanar_times(c, -eps, __dadd_rn(1.0, eps), ts);
    double t_prev = 0.0;
    for (int k = 0; k < nt; ++k) {
      const double t = ts[k];
      d3 Xt[4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
        Xt[a] = d3{__dadd_rn(X[a].x, __dmul_rn(t, P[a].x)), __dadd_rn(X[a].y, __dmul_rn(t, P[a].y)),
                   __dadd_rn(X[a].z, __dmul_rn(t, P[a].z))};
      const Region Rt = ee ? classify_ee(Xt) : classify_pt(Xt);
      const double d = region_distance(Xt, Rt);
      if (d < thr) {
        const double t_ref = __dmul_rn(0.5, __dadd_rn(fmax(t_prev, 0.0), fmax(t, 0.0)));
        const double f_ref = cubic_at(c, t_ref);
        double tr = fmax(t, 0.0);
        for (int it = 0; it < 64; ++it) {
          const double ft = cubic_at(c, tr);
          if (ft != 0.0 && (ft > 0) == (f_ref > 0)) break;
          tr = __dmul_rn(tr, 0.9);
        }
        amin = fmin(amin, fmin(1.0, __dmul_rn(eta_margin, tr)));
        break;
      }
      t_prev = t;
    }
  }
  amin = block_min<double, NT>(amin, 1.0);
  if (threadIdx.x == 0) partials[blockIdx.x] = amin;
}

// keeps a line-search candidate if it can enter A along the step (d < dhat +
// Delta) or can constrain the step length (eta d < Delta); Delta = max |p_a - p_b|
__global__ void k_ls_filter(Dev S, const double* __restrict__ x, const double* __restrict__ dir,
                            const uint64_t* __restrict__ cand, int64_t nc, double eta,
                            uint8_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    Region R;
    const uint64_t key = cand[i];
    const double d = pair_distance(S, x, key, v, X, R);
    d3 P[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) P[a] = ld3(dir, v[a]);
    const int na = key_kind(key) == 0 ? 1 : 2;
    double Dl = 0.0;
    for (int a = 0; a < na; ++a)
      for (int b = na; b < 4; ++b) {
        const d3 w = P[a] - P[b];
        Dl = fmax(Dl, sqrt(dot(w, w)));
      }
    flag[i] = (d < S.dhat + Dl || eta * d < Dl) ? 1 : 0;
  }
}

__global__ void k_flag_below(const double* __restrict__ d, int64_t n, double thr, uint8_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = d[i] < thr ? 1 : 0;
}

__global__ void k_dual_update(Dev S, const double* __restrict__ x, const uint64_t* __restrict__ keys,
                              double* __restrict__ mu, int64_t n, double sigma) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    Region R;
    const double d = pair_distance(S, x, keys[i], v, X, R);
    const double m = mu[i];
    const double s = fmax(-m / sigma - S.dhat + d, 0.0);
    mu[i] = m + sigma * bar(d, S.dhat + s);
  }
}

}  // namespace

bal_status launch_pair_distance(Scene& S, const double* x, const uint64_t* keys, int64_t n,
                                double* d, cudaStream_t st) {
  if (n <= 0) return BAL_OK;
  k_pair_distance<<<grid_for(n), kThreads, 0, st>>>(S.d, x, keys, n, d);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_contact_terms(Scene& S, const double* x, double* grad, bool hess,
                                cudaStream_t st) {
  // friction lagged at x: on for the projected (time-step) Hessian, off for the
  // sigma0 evaluation and the adjoint
  const bool fric = S.prm.friction > 0.0 && S.project && !S.fric_suspend;
  if (fric) S.n_fr = 0;
  if (S.n_eval <= 0) return BAL_OK;
  ContactArgs A;
  A.keys = S.eval_keys.as<uint64_t>();
  A.flags = S.eval_flags.as<uint8_t>();
  A.mu = S.eval_mu.as<double>();
  A.s = S.eval_s.as<double>();
  A.n = S.n_eval;
  A.sigma = S.sigma;
  A.grad = grad;
  A.hess = hess ? 1 : 0;
  A.project = S.project ? 1 : 0;
  if (hess) {
    BAL_TRY(buf_reserve(S.emit_keys, sizeof(uint64_t) * 6 * S.n_eval));
    BAL_TRY(buf_reserve(S.emit_vals, sizeof(double) * 54 * S.n_eval));
  }
  A.emit_keys = S.emit_keys.as<uint64_t>();
  A.emit_vals = S.emit_vals.as<double>();
  A.fric = fric ? 1 : 0;
  A.chi = S.prm.friction;
  A.eps_h = (S.prm.friction_eps_v > 0.0 ? S.prm.friction_eps_v : S.d.dhat) * S.d.h;
  A.xt = S.xt;
  A.fr_beta = A.fr_n = A.fr_lam = nullptr;
  if (A.fric) {
    BAL_TRY(buf_reserve(S.fr_keys, sizeof(uint64_t) * (S.n_eval + 1)));
    BAL_TRY(buf_reserve(S.fr_beta, sizeof(double) * 4 * (S.n_eval + 1)));
    BAL_TRY(buf_reserve(S.fr_n, sizeof(double) * 3 * (S.n_eval + 1)));
    BAL_TRY(buf_reserve(S.fr_lam, sizeof(double) * (S.n_eval + 1)));
    BAL_CUDA(cudaMemcpyAsync(S.fr_keys.p, S.eval_keys.p, sizeof(uint64_t) * S.n_eval,
                             cudaMemcpyDeviceToDevice, st));
    A.fr_beta = S.fr_beta.as<double>();
    A.fr_n = S.fr_n.as<double>();
    A.fr_lam = S.fr_lam.as<double>();
    S.n_fr = S.n_eval;
  }
  k_contact_terms<<<grid_for(S.n_eval, 128, kNumSM * 8), 128, 0, st>>>(S.d, x, A);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_contact_energy(Scene& S, const double* x, const uint64_t* cand, int64_t ncand,
                                 int slot, cudaStream_t st) {
  constexpr int NT = 256;
  const int nblk = 2 * kNumSM;
  const int64_t nap = (int64_t)S.ap_keys.size();
  FricLag F;
  F.keys = S.fr_keys.as<uint64_t>();
  F.beta = S.fr_beta.as<double>();
  F.nrm = S.fr_n.as<double>();
  F.lam = S.fr_lam.as<double>();
  F.xt = S.xt;
  F.n = S.prm.friction > 0.0 ? S.n_fr : 0;
  F.chi = S.prm.friction;
  F.eps_h = (S.prm.friction_eps_v > 0.0 ? S.prm.friction_eps_v : S.d.dhat) * S.d.h;
  k_contact_energy<NT><<<nblk, NT, 0, st>>>(S.d, x, cand, ncand, S.ap_keys_d.as<uint64_t>(),
                                            S.ap_mu_d.as<double>(), S.ap_s_d.as<double>(), nap,
                                            S.sigma, F, S.partials, nblk);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce_offset(S, 0, nblk, slot, RED_SUM, st));
  BAL_TRY(finish_reduce_offset(S, nblk, nblk, slot + 1, RED_SUM, st));
  return BAL_OK;
}

bal_status launch_step_bound(Scene& S, const double* x, const double* dir,
                             const uint64_t* cand, int64_t ncand, int slot, cudaStream_t st) {
  constexpr int NT = 256;
  const int nblk = 2 * kNumSM;
  k_step_bound<NT><<<nblk, NT, 0, st>>>(S.d, x, dir, cand, ncand, S.prm.step_bound,
                                        S.prm.ca_max_iter > 0 ? S.prm.ca_max_iter : 64, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return finish_reduce(S, nblk, slot, RED_MIN, st);
}

bal_status launch_ccd_bound(Scene& S, const double* x, const double* dir, const uint64_t* cand,
                            int64_t ncand, int slot, cudaStream_t st) {
  constexpr int NT = 256;
  const int nblk = 2 * kNumSM;
  k_ccd_toi<NT><<<nblk, NT, 0, st>>>(S.d, x, dir, cand, ncand, S.prm.step_bound, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return finish_reduce(S, nblk, slot, RED_MIN, st);
}

bal_status launch_ls_filter(Scene& S, const double* x, const double* dir, const uint64_t* cand,
                            int64_t n, uint8_t* flag, cudaStream_t st) {
  if (n <= 0) return BAL_OK;
  k_ls_filter<<<grid_for(n), kThreads, 0, st>>>(S.d, x, dir, cand, n, S.prm.step_bound, flag);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_flag_below(const double* d, int64_t n, double thr, uint8_t* flag, cudaStream_t st) {
  if (n <= 0) return BAL_OK;
  k_flag_below<<<grid_for(n), kThreads, 0, st>>>(d, n, thr, flag);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_dual_update(Scene& S, const double* x, int64_t n, cudaStream_t st) {
  if (n <= 0) return BAL_OK;
  k_dual_update<<<grid_for(n), kThreads, 0, st>>>(S.d, x, S.ap_keys_d.as<uint64_t>(),
                                                 S.ap_mu_d.as<double>(), n, S.sigma);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

}  // namespace bal
