// Small FP64 vector kernels of the Newton loop: inertia target, axpy, dot
// products (deterministic two-stage sums), per-vertex step length, velocity.
#include "scene.cuh"

namespace bal {

namespace {

constexpr int kRB = 2 * kNumSM;

// y = x_t + h v_t + h^2 g (Sec. 3.1); pinned vertices keep y = x_t.
__global__ void k_make_y(Dev S, const double* __restrict__ xt, const double* __restrict__ vt,
                         double gx, double gy, double gz, double* __restrict__ y) {
  const double h = S.h, h2 = S.h * S.h;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    const d3 x = ld3(xt, v);
    st3(y, v, S.pinned[v] ? x : x + h * ld3(vt, v) + d3{h2 * gx, h2 * gy, h2 * gz});
  }
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, const double* __restrict__ y,
                       double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y[i] + a * x[i];
}

template <int NT>
__global__ void __launch_bounds__(NT) k_dot(int64_t n, const double* __restrict__ a,
                                            const double* __restrict__ b, double* partials) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    s += a[i] * b[i];
  s = block_sum<double, NT>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_surf_max_norm(Dev S, const double* __restrict__ d,
                                                      double* partials) {
  double m = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < S.nsv; i += gridDim.x * NT) {
    const d3 v = ld3(d, S.surf[i]);
    m = fmax(m, sqrt(dot(v, v)));
  }
  m = block_max<double, NT>(m, 0.0);
  if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

// max and min of the assembled eigenvalue stiffness Lambda over free DOFs
// (App. B condition-number estimate): partials [0, nb) max, [nb, 2 nb) min
template <int NT>
__global__ void __launch_bounds__(NT) k_lambda_range(Dev S, double* partials, int nb) {
  double hi = 0.0, lo = INFINITY;
  for (int v = blockIdx.x * NT + threadIdx.x; v < S.nv; v += gridDim.x * NT) {
    if (S.pinned[v]) continue;
    const d3 l = ld3(S.Lambda, v);
    hi = fmax(hi, fmax(l.x, fmax(l.y, l.z)));
    lo = fmin(lo, fmin(l.x, fmin(l.y, l.z)));
  }
  hi = block_max<double, NT>(hi, 0.0);
  lo = block_min<double, NT>(lo, INFINITY);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = hi;
    partials[nb + blockIdx.x] = lo;
  }
}

}  // namespace

bal_status launch_lambda_range(Scene& S, int slot, cudaStream_t st) {
  k_lambda_range<256><<<kRB, 256, 0, st>>>(S.d, S.partials, kRB);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(finish_reduce_offset(S, 0, kRB, slot, RED_MAX, st));
  return finish_reduce_offset(S, kRB, kRB, slot + 1, RED_MIN, st);
}

bal_status launch_make_y(Scene& S, const double* xt, const double* vt, double* y, cudaStream_t st) {
  k_make_y<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, xt, vt, S.grav[0], S.grav[1], S.grav[2], y);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_axpy(Scene& S, int64_t n, double a, const double* x, const double* y, double* out,
                       cudaStream_t st) {
  k_axpy<<<grid_for(n), kThreads, 0, st>>>(n, a, x, y, out);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status launch_dot(Scene& S, int64_t n, const double* a, const double* b, int slot, cudaStream_t st) {
  k_dot<256><<<kRB, 256, 0, st>>>(n, a, b, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return finish_reduce(S, kRB, slot, RED_SUM, st);
}

bal_status launch_surf_max_norm(Scene& S, const double* d, int slot, cudaStream_t st) {
  k_surf_max_norm<256><<<kRB, 256, 0, st>>>(S.d, d, S.partials);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return finish_reduce(S, kRB, slot, RED_MAX, st);
}

}  // namespace bal
