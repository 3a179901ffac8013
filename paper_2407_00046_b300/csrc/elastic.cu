// Neo-Hookean tetrahedral elasticity and inertia (Sec. 3.1) on the GPU: FP64,
// with the element stencil Hessians optionally in FP32 (single-precision path).
//
// Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2 (the NH of IPC; the
// paper names the model only). The element stencil Hessian is projected to PSD
// in deformation-gradient space (Sec. 4.2.2): the 9x9 dP/dF of an isotropic
// energy decomposes, in the rotated basis U E_ij V^T of the signed SVD
// F = U diag(s) V^T, into
//   - a 3x3 "scaling" block  d2Psi/ds_i ds_j  = diag(mu + (mu - lam lnJ)/s_i^2)
//                                               + lam (1/s)(1/s)^T,
//   - per pair (i,j) a "flip" mode  U (E_ij + E_ji) V^T / sqrt2 with eigenvalue
//     mu + (mu - lam lnJ)/(s_i s_j), and a "twist" mode U (E_ij - E_ji) V^T /
//     sqrt2 with eigenvalue mu - (mu - lam lnJ)/(s_i s_j),
// (analytic eigensystems of isotropic distortion energies, Smith et al. 2019,
// restated for this energy). Only positive modes are kept, so the projected
// 12x12 block is V_e sum_k lambda_k^+ w_k w_k^T with w_k = d vec(F)/dx ^T vec(D_k).
// Rigid translations are in the null space, so only the 9x9 sub-block of
// vertices 1..3 is accumulated; the blocks touching vertex 0 follow by sums.
#include <cub/cub.cuh>

#include "scene.cuh"

namespace bal {

namespace {

__device__ inline void load_tet(const Dev& S, const double* __restrict__ x, int t, int v[4],
                                d3 X[4]) {
  const int4 tv = reinterpret_cast<const int4*>(S.tets)[t];
  v[0] = tv.x; v[1] = tv.y; v[2] = tv.z; v[3] = tv.w;
#pragma unroll
  for (int a = 0; a < 4; ++a) X[a] = ld3(x, v[a]);
}

// F = Ds Dm^{-1}, Ds columns x_{a+1} - x_0.
__device__ inline void def_grad(const d3 X[4], const double* __restrict__ Mi, double F[3][3]) {
  const d3 e[3] = {X[1] - X[0], X[2] - X[0], X[3] - X[0]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double ei[3] = {i == 0 ? e[0].x : (i == 1 ? e[0].y : e[0].z),
                          i == 0 ? e[1].x : (i == 1 ? e[1].y : e[1].z),
                          i == 0 ? e[2].x : (i == 1 ? e[2].y : e[2].z)};
#pragma unroll
    for (int j = 0; j < 3; ++j) F[i][j] = ei[0] * Mi[j] + ei[1] * Mi[3 + j] + ei[2] * Mi[6 + j];
  }
}

__device__ inline double det3(const double F[3][3]) {
  return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
         F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}

// F = Ds Dm^{-1} in arithmetic T: the edge vectors x_{a+1} - x_0 are formed in
// FP64 (absolute coordinates would cancel in FP32), then rounded to T.
template <typename T>
__device__ inline void def_grad_t(const d3 X[4], const double* __restrict__ Mi, T F[3][3]) {
  const d3 e[3] = {X[1] - X[0], X[2] - X[0], X[3] - X[0]};
  T m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = (T)Mi[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T ei[3] = {(T)(i == 0 ? e[0].x : (i == 1 ? e[0].y : e[0].z)),
                     (T)(i == 0 ? e[1].x : (i == 1 ? e[1].y : e[1].z)),
                     (T)(i == 0 ? e[2].x : (i == 1 ? e[2].y : e[2].z))};
#pragma unroll
    for (int j = 0; j < 3; ++j) F[i][j] = ei[0] * m[j] + ei[1] * m[3 + j] + ei[2] * m[6 + j];
  }
}

// squared relative off-diagonal size at which the 3x3 Jacobi iteration stops
template <typename T> struct JacobiTol;
template <> struct JacobiTol<double> { static constexpr double v = 1e-34; };
template <> struct JacobiTol<float> { static constexpr float v = 1e-14f; };

// Cyclic Jacobi for a symmetric 3x3 (in place). A ends (nearly) diagonal; V
// holds the eigenvectors in its columns.
template <typename T>
__device__ inline void jacobi3(T A[3][3], T V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const T off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const T dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= JacobiTol<T>::v * dia || off == T(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const T apq = A[p][q];
      if (apq == T(0)) continue;
      const T theta = (A[q][q] - A[p][p]) / (T(2) * apq);
      const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
      const T c = T(1) / sqrt(t * t + T(1)), s = t * c;
      const int r = 3 - p - q;
      const T arp = A[r][p], arq = A[r][q];
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = T(0);
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
}

// Signed SVD F = U diag(s) V^T with det U = det V = +1, s descending in
// magnitude; s[2] carries the sign of det F.
template <typename T>
__device__ inline void svd3(const T F[3][3], T U[3][3], T s[3], T V[3][3]) {
  T C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  jacobi3<T>(C, V);
  T w[3] = {C[0][0], C[1][1], C[2][2]};
  // sort descending (swap columns of V)
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (w[i] < w[i + 1]) {
        const T tw = w[i]; w[i] = w[i + 1]; w[i + 1] = tw;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T tv = V[k][i]; V[k][i] = V[k][i + 1]; V[k][i + 1] = tv;
        }
      }
    }
  }
  const T dV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
               V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
               V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (dV < T(0)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
  }
  // columns of F V; U by Gram-Schmidt on the first two, the third by a cross product
  T Fv[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < 3; ++i) Fv[c][i] = F[i][0] * V[0][c] + F[i][1] * V[1][c] + F[i][2] * V[2][c];
  const T n0 = T(1) / sqrt(Fv[0][0] * Fv[0][0] + Fv[0][1] * Fv[0][1] + Fv[0][2] * Fv[0][2]);
  T u0[3], t1[3], u1[3], u2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) u0[i] = n0 * Fv[0][i];
  const T p01 = u0[0] * Fv[1][0] + u0[1] * Fv[1][1] + u0[2] * Fv[1][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) t1[i] = Fv[1][i] - p01 * u0[i];
  const T n1 = T(1) / sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) u1[i] = n1 * t1[i];
  u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
  u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
  u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
  s[0] = u0[0] * Fv[0][0] + u0[1] * Fv[0][1] + u0[2] * Fv[0][2];
  s[1] = u1[0] * Fv[1][0] + u1[1] * Fv[1][1] + u1[2] * Fv[1][2];
  s[2] = u2[0] * Fv[2][0] + u2[1] * Fv[2][1] + u2[2] * Fv[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    U[i][0] = u0[i];
    U[i][1] = u1[i];
    U[i][2] = u2[i];
  }
}

// H (upper triangle of a symmetric 9x9, row-major packed 45) += lam w w^T
template <typename T>
__device__ inline void rank1_45(T H[45], const T w[9], T lam) {
  int k = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T li = lam * w[i];
#pragma unroll
    for (int j = i; j < 9; ++j) H[k++] += li * w[j];
  }
}
template <typename T>
__device__ inline T h45(const T H[45], int i, int j) {
  if (i > j) { const int t = i; i = j; j = t; }
  return H[i * 9 - (i * (i - 1)) / 2 + (j - i)];
}

__global__ void k_inertia_grad(Dev S, const double* __restrict__ x, double* __restrict__ g) {
  const double ih2 = 1.0 / (S.h * S.h);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    if (S.pinned[v]) {
      st3(g, v, d3{0, 0, 0});
    } else {
      const double m = S.mass[v] * ih2;
      st3(g, v, m * (ld3(x, v) - ld3(S.y, v)));
    }
  }
}

__global__ void k_elastic_grad(Dev S, const double* __restrict__ x, double* __restrict__ g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.nt; t += gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    load_tet(S, x, t, v, X);
    const double* Mi = S.Dm_inv + 9 * (int64_t)t;
    double F[3][3];
    def_grad(X, Mi, F);
    const double J = det3(F);
    const double mu = S.mu[t], lam = S.lam[t], vol = S.vol[t];
    const double lnJ = log(J);
    // F^{-T} = cof(F) / J
    double A[3][3];
    A[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) / J;
    A[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) / J;
    A[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) / J;
    A[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) / J;
    A[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) / J;
    A[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) / J;
    A[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) / J;
    A[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) / J;
    A[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) / J;
    double P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) P[i][j] = mu * (F[i][j] - A[i][j]) + lam * lnJ * A[i][j];
    d3 gs = d3{0, 0, 0};
#pragma unroll
    for (int b = 1; b < 4; ++b) {
      const double* B = Mi + 3 * (b - 1);
      d3 gb = d3{vol * (P[0][0] * B[0] + P[0][1] * B[1] + P[0][2] * B[2]),
                 vol * (P[1][0] * B[0] + P[1][1] * B[1] + P[1][2] * B[2]),
                 vol * (P[2][0] * B[0] + P[2][1] * B[1] + P[2][2] * B[2])};
      gs = gs + gb;
      if (!S.pinned[v[b]]) atomic_add3(g, v[b], gb);
    }
    if (!S.pinned[v[0]]) atomic_add3(g, v[0], -gs);
  }
}

__global__ void k_assemble_init(Dev S) {
  const double ih2 = 1.0 / (S.h * S.h);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    const double m = S.mass[v] * ih2;
    double* D = S.D + 9 * (int64_t)v;
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = (k % 4 == 0) ? m : 0.0;
    S.Lambda[3 * v] = m;
    S.Lambda[3 * v + 1] = m;
    S.Lambda[3 * v + 2] = m;
  }
}

template <typename T>
__device__ inline void add_block(double* dst, const T blk[3][3], bool transpose) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(dst + 3 * i + k, (double)(transpose ? blk[k][i] : blk[i][k]));
}

// Element stencil Hessians in arithmetic T (double: the FP64 path; float: the
// single-precision path), accumulated into the FP64 block storage.
template <typename T>
__global__ void __launch_bounds__(128) k_elastic_hess(Dev S, const double* __restrict__ x, int project) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.nt; t += gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    load_tet(S, x, t, v, X);
    const double* Md = S.Dm_inv + 9 * (int64_t)t;
    T F[3][3], Mi[9];
    def_grad_t<T>(X, Md, F);
#pragma unroll
    for (int k = 0; k < 9; ++k) Mi[k] = (T)Md[k];
    const T mu = (T)S.mu[t], lam = (T)S.lam[t], vol = (T)S.vol[t];
    T U[3][3], s[3], V[3][3];
    svd3<T>(F, U, s, V);
    const T lnJ = log(s[0] * s[1] * s[2]);
    const T c = mu - lam * lnJ;
    // beta[b][m] = v_m . B_b  (B_b = row b-1 of Dm^{-1}, b = 1..3)
    T beta[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        beta[b][m] = V[0][m] * Mi[3 * b] + V[1][m] * Mi[3 * b + 1] + V[2][m] * Mi[3 * b + 2];
    T H[45];
#pragma unroll
    for (int k = 0; k < 45; ++k) H[k] = T(0);
    T w[9];
    // scaling modes: eigen-decomposition of diag(mu + c/s^2) + lam (1/s)(1/s)^T
    {
      T A[3][3], Q[3][3];
      const T is[3] = {T(1) / s[0], T(1) / s[1], T(1) / s[2]};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          A[i][j] = lam * is[i] * is[j] + (i == j ? mu + c * is[i] * is[i] : T(0));
      jacobi3<T>(A, Q);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T ev = A[k][k];
        if (project && ev <= T(0)) continue;
        // w[b][i] = sum_m U[i][m] q_m beta[b][m]
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const T c0 = Q[0][k] * beta[b][0], c1 = Q[1][k] * beta[b][1], c2 = Q[2][k] * beta[b][2];
#pragma unroll
          for (int i = 0; i < 3; ++i) w[3 * b + i] = U[i][0] * c0 + U[i][1] * c1 + U[i][2] * c2;
        }
        rank1_45<T>(H, w, ev);
      }
    }
    // flip / twist modes of each singular-value pair
    const T r2 = (T)0.70710678118654752440;
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
      const int i = pr == 2 ? 1 : 0;
      const int j = pr == 0 ? 1 : 2;
      const T q = c / (s[i] * s[j]);
#pragma unroll
      for (int sgn = 0; sgn < 2; ++sgn) {
        const T ev = sgn == 0 ? mu + q : mu - q;   // flip : twist
        if (project && ev <= T(0)) continue;
        const T sg = sgn == 0 ? T(1) : T(-1);
        // D = U (E_ij +- E_ji) V^T / sqrt2 ; w[b] = (u_i beta_bj +- u_j beta_bi)/sqrt2
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const T ci = r2 * beta[b][j], cj = sg * r2 * beta[b][i];
#pragma unroll
          for (int k = 0; k < 3; ++k) w[3 * b + k] = U[k][i] * ci + U[k][j] * cj;
        }
        rank1_45<T>(H, w, ev);
      }
    }
    // blocks of vertices 1..3, scaled by the rest volume
    T blk[4][4][3][3];
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int b = 1; b < 4; ++b)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) blk[a][b][i][k] = vol * h45<T>(H, 3 * (a - 1) + i, 3 * (b - 1) + k);
    // translation invariance: H[a][0] = -sum_b H[a][b], H[0][0] = sum_ab H[a][b]
#pragma unroll
    for (int a = 1; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T sum = blk[a][1][i][k] + blk[a][2][i][k] + blk[a][3][i][k];
          blk[a][0][i][k] = -sum;
          blk[0][a][k][i] = -sum;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) blk[0][0][i][k] = -(blk[1][0][i][k] + blk[2][0][i][k] + blk[3][0][i][k]);
    // the two summation orders of H[0][0] round differently: keep the block symmetric
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = i + 1; k < 3; ++k) {
        const T m = T(0.5) * (blk[0][0][i][k] + blk[0][0][k][i]);
        blk[0][0][i][k] = m;
        blk[0][0][k][i] = m;
      }
    // Lambda: mean eigenvalue of the projected element stencil = trace / 12
    T trT = T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) trT += blk[a][a][0][0] + blk[a][a][1][1] + blk[a][a][2][2];
    const double tr = (double)trT * (1.0 / 12.0);
    bool pin[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      pin[a] = S.pinned[v[a]] != 0;
      atomicAdd(S.Lambda + 3 * v[a], tr);
      atomicAdd(S.Lambda + 3 * v[a] + 1, tr);
      atomicAdd(S.Lambda + 3 * v[a] + 2, tr);
      if (!pin[a]) add_block<T>(S.D + 9 * (int64_t)v[a], blk[a][a], false);
    }
    const int pa[6] = {1, 2, 3, 2, 3, 3};
    const int pb[6] = {0, 0, 0, 1, 1, 2};
    const int* slots = S.tet_slot + 6 * (int64_t)t;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int a = pa[k], b = pb[k];
      if (pin[a] || pin[b]) continue;
      const int code = slots[k];
      add_block<T>(S.Lval + 9 * (int64_t)(code >> 1), blk[a][b], (code & 1) != 0);
    }
  }
}

// dJ/dE_e += -lambda_e^T (d grad W_e / d E_e) = -lambda_e^T grad W_e / E_e
// (mu and lam are linear in E); pinned DOFs of lambda are zero.
__global__ void k_dLdE(Dev S, const double* __restrict__ x, const double* __restrict__ lam_adj,
                       const double* __restrict__ E, double* __restrict__ acc) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.nt; t += gridDim.x * blockDim.x) {
    int v[4];
    d3 X[4];
    load_tet(S, x, t, v, X);
    const double* Mi = S.Dm_inv + 9 * (int64_t)t;
    double F[3][3];
    def_grad(X, Mi, F);
    const double J = det3(F);
    const double mu = S.mu[t], lam = S.lam[t], vol = S.vol[t];
    const double lnJ = log(J);
    double A[3][3];
    A[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) / J;
    A[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) / J;
    A[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) / J;
    A[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) / J;
    A[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) / J;
    A[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) / J;
    A[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) / J;
    A[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) / J;
    A[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) / J;
    double P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) P[i][j] = mu * (F[i][j] - A[i][j]) + lam * lnJ * A[i][j];
    d3 gs = d3{0, 0, 0};
    double dot_acc = 0.0;
#pragma unroll
    for (int b = 1; b < 4; ++b) {
      const double* B = Mi + 3 * (b - 1);
      d3 gb = d3{vol * (P[0][0] * B[0] + P[0][1] * B[1] + P[0][2] * B[2]),
                 vol * (P[1][0] * B[0] + P[1][1] * B[1] + P[1][2] * B[2]),
                 vol * (P[2][0] * B[0] + P[2][1] * B[1] + P[2][2] * B[2])};
      gs = gs + gb;
      dot_acc += dot(ld3(lam_adj, v[b]), gb);
    }
    dot_acc += dot(ld3(lam_adj, v[0]), -gs);
    acc[t] -= dot_acc / E[t];
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_energy(Dev S, const double* __restrict__ x,
                                               double* __restrict__ partials, int nblk) {
  double ein = 0.0, eel = 0.0, ninv = 0.0;
  const double ih2 = 0.5 / (S.h * S.h);
  for (int v = blockIdx.x * NT + threadIdx.x; v < S.nv; v += gridDim.x * NT) {
    if (!S.pinned[v]) {
      const d3 r = ld3(x, v) - ld3(S.y, v);
      ein += ih2 * S.mass[v] * dot(r, r);
    }
  }
  for (int t = blockIdx.x * NT + threadIdx.x; t < S.nt; t += gridDim.x * NT) {
    int v[4];
    d3 X[4];
    load_tet(S, x, t, v, X);
    double F[3][3];
    def_grad(X, S.Dm_inv + 9 * (int64_t)t, F);
    const double J = det3(F);
    if (!(J > 0.0)) {
      ninv += 1.0;
      continue;
    }
    const double lnJ = log(J);
    double I1 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) I1 += F[i][j] * F[i][j];
    const double mu = S.mu[t], lam = S.lam[t];
    eel += S.vol[t] * (0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
  }
  ein = block_sum<double, NT>(ein);
  eel = block_sum<double, NT>(eel);
  ninv = block_sum<double, NT>(ninv);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = ein;
    partials[nblk + blockIdx.x] = eel;
    partials[2 * nblk + blockIdx.x] = ninv;
  }
}

}  // namespace

bal_status launch_inertia_elastic_grad(Scene& S, const double* x, double* grad, cudaStream_t st) {
  k_inertia_grad<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, x, grad);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  k_elastic_grad<<<grid_for(S.d.nt), kThreads, 0, st>>>(S.d, x, grad);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_elastic_assemble(Scene& S, const double* x, cudaStream_t st) {
  k_assemble_init<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  if (S.d.nnzL > 0) BAL_CUDA(cudaMemsetAsync(S.d.Lval, 0, sizeof(double) * 9 * S.d.nnzL, st));
  if (S.d.nt > 0) {
    // single-precision path: element eigensystems in FP32 (projected Hessian only)
    if (S.ktime) cudaEventRecord(S.kaev[0], st);
    if (S.prm.precision == BAL_PREC_FP32 && S.project)
      k_elastic_hess<float><<<grid_for(S.d.nt, 128, kNumSM * 32), 128, 0, st>>>(S.d, x, 1);
    else
      k_elastic_hess<double><<<grid_for(S.d.nt, 128, kNumSM * 32), 128, 0, st>>>(S.d, x, S.project ? 1 : 0);
    if (S.ktime) cudaEventRecord(S.kaev[1], st);
    ::bal::note_launch();
    BAL_LAUNCH_CHECK();
  }
  return BAL_OK;
}

bal_status launch_dLdE(Scene& S, const double* x, const double* lam_adj, double* acc, cudaStream_t st) {
  k_dLdE<<<grid_for(S.d.nt), kThreads, 0, st>>>(S.d, x, lam_adj, S.E, acc);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_elastic_energy(Scene& S, const double* x, cudaStream_t st) {
  constexpr int NT = 256;
  const int nblk = 2 * kNumSM;
  k_energy<NT><<<nblk, NT, 0, st>>>(S.d, x, S.partials, nblk);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce(S, nblk, 0, RED_SUM, st));
  BAL_TRY(finish_reduce_offset(S, nblk, nblk, 1, RED_SUM, st));
  BAL_TRY(finish_reduce_offset(S, 2 * nblk, nblk, 2, RED_SUM, st));
  return BAL_OK;
}

}  // namespace bal
