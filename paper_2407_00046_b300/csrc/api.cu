// C ABI of libbal: scene lifetime, time-step state and the Algorithm 1 driver.
//
// The host drives the primal-dual loop of Algorithm 1 (Sec. 3.3) and makes the
// discrete decisions (A' rule, sigma schedule, convergence, line-search
// acceptance) from scalars the kernels reduce on the device; every array
// operation runs in the CUDA kernels of this library.
#include <atomic>
#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "scene.cuh"

struct bal_scene {
  bal::Scene S;
};

namespace bal {

// ---- errors --------------------------------------------------------------------
static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

bal_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what,
            file, line);
  return BAL_ERR_CUDA;
}

bal_status kt_collect(Scene& S, int n) {
  if (!S.ktime) return BAL_OK;
  for (int k = 0; k < n; ++k) {
    float ms = 0.f;
    BAL_CUDA(cudaEventElapsedTime(&ms, S.kev[2 * k], S.kev[2 * k + 1]));
    S.kt_ms += ms;
    S.kt_n += 1;
  }
  return BAL_OK;
}

bal_status buf_reserve(Buf& b, size_t bytes) {
  if (bytes <= b.cap && b.p) return BAL_OK;
  if (b.p) {
    BAL_CUDA(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes < 256 ? 256 : bytes;
  want = want + want / 8;
  BAL_CUDA(cudaMalloc(&b.p, want));
  b.cap = want;
  return BAL_OK;
}

void buf_free(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

namespace {

using clk = std::chrono::steady_clock;
inline double ms_since(clk::time_point t0) {
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

template <typename T>
bal_status dalloc(Scene& S, T** p, size_t n) {
  void* q = nullptr;
  BAL_CUDA(cudaMalloc(&q, sizeof(T) * (n > 0 ? n : 1)));
  S.owned.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return BAL_OK;
}
template <typename T>
bal_status dupload(Scene& S, const T** p, const T* host, size_t n) {
  T* q = nullptr;
  BAL_TRY(dalloc(S, &q, n));
  if (n) BAL_CUDA(cudaMemcpy(q, host, sizeof(T) * n, cudaMemcpyHostToDevice));
  *p = q;
  return BAL_OK;
}

bal_status read_scalars(Scene& S, double* out, int first, int count, cudaStream_t st) {
  BAL_CUDA(cudaMemcpyAsync(out, S.scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}

inline double barrier_b(double d, double c) {
  if (!(d > 0.0)) return INFINITY;
  if (d >= c) return 0.0;
  return -(d - c) * (d - c) * std::log(d / c);
}
inline double barrier_d2b(double d, double c) {
  if (!(d > 0.0) || d >= c) return 0.0;
  const double t = d - c;
  return -2.0 * std::log(d / c) - 4.0 * t / d + t * t / (d * d);
}

// A at x: candidates within dhat, exact distances, keep d < dhat (compacted on
// the device; host copies of A only).
bal_status detect_active(Scene& S, const double* x, std::vector<uint64_t>& keys,
                         std::vector<double>& dist, cudaStream_t st) {
  BAL_TRY(find_candidates(S, x, S.d.dhat, S.cand, S.cand_alt, &S.n_cand, st));
  keys.clear();
  dist.clear();
  if (S.n_cand == 0) return BAL_OK;
  const int64_t n = S.n_cand;
  BAL_TRY(buf_reserve(S.dist, sizeof(double) * n));
  BAL_TRY(buf_reserve(S.dist_alt, sizeof(double) * n));
  BAL_TRY(buf_reserve(S.flags, n));
  BAL_TRY(buf_reserve(S.cand_alt, sizeof(uint64_t) * n));
  BAL_TRY(launch_pair_distance(S, x, S.cand.as<uint64_t>(), n, S.dist.as<double>(), st));
  BAL_TRY(launch_flag_below(S.dist.as<double>(), n, S.d.dhat, S.flags.as<uint8_t>(), st));
  int64_t na = 0, nd = 0;
  BAL_TRY(compact_u64(S, S.cand.as<uint64_t>(), S.flags.as<uint8_t>(), n, S.cand_alt.as<uint64_t>(),
                      &na, st));
  BAL_TRY(compact_f64(S, S.dist.as<double>(), S.flags.as<uint8_t>(), n, S.dist_alt.as<double>(), &nd,
                      st));
  keys.resize(na);
  dist.resize(na);
  if (na) {
    BAL_CUDA(cudaMemcpyAsync(keys.data(), S.cand_alt.p, sizeof(uint64_t) * na, cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaMemcpyAsync(dist.data(), S.dist_alt.p, sizeof(double) * na, cudaMemcpyDeviceToHost, st));
    BAL_CUDA(cudaStreamSynchronize(st));
  }
  return BAL_OK;
}

// Upload A' (keys, mu) to the device.
bal_status upload_ap(Scene& S, cudaStream_t st) {
  const size_t n = S.ap_keys.size();
  BAL_TRY(buf_reserve(S.ap_keys_d, sizeof(uint64_t) * (n + 1)));
  BAL_TRY(buf_reserve(S.ap_mu_d, sizeof(double) * (n + 1)));
  BAL_TRY(buf_reserve(S.ap_s_d, sizeof(double) * (n + 1)));
  if (n) {
    BAL_CUDA(cudaMemcpyAsync(S.ap_keys_d.p, S.ap_keys.data(), sizeof(uint64_t) * n,
                             cudaMemcpyHostToDevice, st));
    BAL_CUDA(cudaMemcpyAsync(S.ap_mu_d.p, S.ap_mu.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  return BAL_OK;
}

// Evaluation list A u A' with flags, mu and s_i = max(-mu/sigma - dhat + d, 0)
// evaluated at x (Sec. 3.2.2); also fills the device A' slack used by the line
// search energy.
bal_status build_eval(Scene& S, const double* x, const std::vector<uint64_t>& A_keys,
                      cudaStream_t st) {
  std::vector<uint64_t> keys;
  std::vector<uint8_t> flags;
  std::vector<double> mu;
  keys.reserve(A_keys.size() + S.ap_keys.size());
  size_t i = 0, j = 0;
  while (i < A_keys.size() || j < S.ap_keys.size()) {
    if (j >= S.ap_keys.size() || (i < A_keys.size() && A_keys[i] < S.ap_keys[j])) {
      keys.push_back(A_keys[i++]);
      flags.push_back(PF_A);
      mu.push_back(0.0);
    } else if (i >= A_keys.size() || S.ap_keys[j] < A_keys[i]) {
      keys.push_back(S.ap_keys[j]);
      flags.push_back(PF_AP);
      mu.push_back(S.ap_mu[j++]);
    } else {
      keys.push_back(A_keys[i++]);
      flags.push_back(PF_A | PF_AP);
      mu.push_back(S.ap_mu[j++]);
    }
  }
  const int64_t n = (int64_t)keys.size();
  S.n_eval = n;
  BAL_TRY(buf_reserve(S.eval_keys, sizeof(uint64_t) * (n + 1)));
  BAL_TRY(buf_reserve(S.eval_flags, n + 1));
  BAL_TRY(buf_reserve(S.eval_mu, sizeof(double) * (n + 1)));
  BAL_TRY(buf_reserve(S.eval_s, sizeof(double) * (n + 1)));
  BAL_TRY(upload_ap(S, st));
  if (n == 0) return BAL_OK;
  BAL_CUDA(cudaMemcpyAsync(S.eval_keys.p, keys.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
  BAL_CUDA(cudaMemcpyAsync(S.eval_flags.p, flags.data(), n, cudaMemcpyHostToDevice, st));
  BAL_CUDA(cudaMemcpyAsync(S.eval_mu.p, mu.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  // distances of the evaluation list -> s
  BAL_TRY(buf_reserve(S.dist, sizeof(double) * n));
  BAL_TRY(launch_pair_distance(S, x, S.eval_keys.as<uint64_t>(), n, S.dist.as<double>(), st));
  std::vector<double> d(n), s(n, 0.0), aps;
  BAL_CUDA(cudaMemcpyAsync(d.data(), S.dist.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  aps.reserve(S.ap_keys.size());
  for (int64_t k = 0; k < n; ++k) {
    if (flags[k] & PF_AP) {
      s[k] = std::max(-mu[k] / S.sigma - S.d.dhat + d[k], 0.0);
      aps.push_back(s[k]);
    }
  }
  BAL_CUDA(cudaMemcpyAsync(S.eval_s.p, s.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (!aps.empty())
    BAL_CUDA(cudaMemcpyAsync(S.ap_s_d.p, aps.data(), sizeof(double) * aps.size(), cudaMemcpyHostToDevice, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}

// gradient of L_sigma at x into g (eval list must be current)
bal_status gradient(Scene& S, const double* x, double* g, cudaStream_t st) {
  BAL_TRY(launch_inertia_elastic_grad(S, x, g, st));
  BAL_TRY(launch_contact_terms(S, x, g, false, st));
  return BAL_OK;
}

// projected Hessian at x (eval list must be current); contact gradient into g if non-null
bal_status assemble(Scene& S, const double* x, double* g, cudaStream_t st) {
  if (S.ktime) BAL_CUDA(cudaEventRecord(S.kaev[2], st));
  BAL_TRY(launch_elastic_assemble(S, x, st));
  BAL_TRY(launch_contact_terms(S, x, g, true, st));
  BAL_TRY(contact_blocks_reduce(S, 6 * S.n_eval, st));
  BAL_TRY(launch_dinv(S, st));
  if (S.ktime) {
    BAL_CUDA(cudaEventRecord(S.kaev[3], st));
    BAL_CUDA(cudaEventSynchronize(S.kaev[3]));
    float e = 0.f, t = 0.f;
    if (S.d.nt > 0) BAL_CUDA(cudaEventElapsedTime(&e, S.kaev[0], S.kaev[1]));
    BAL_CUDA(cudaEventElapsedTime(&t, S.kaev[2], S.kaev[3]));
    S.ka_elastic_ms += e;
    S.ka_total_ms += t;
    S.ka_n += 1;
  }
  S.assembled = true;
  S.f32_valid = false;
  S.dd_valid = false;
  return BAL_OK;
}

// energy parts at x over candidate list cand (barrier for d < dhat) and the
// device A' list: out[0] inertia, out[1] elastic, out[2] contact, out[3] #inverted,
// out[4] #(d < dhat)
bal_status energy_parts(Scene& S, const double* x, const uint64_t* cand, int64_t ncand,
                        double out[5], cudaStream_t st) {
  BAL_TRY(launch_elastic_energy(S, x, st));
  BAL_TRY(launch_contact_energy(S, x, cand, ncand, 4, st));
  double v[6];
  BAL_TRY(read_scalars(S, v, 0, 6, st));
  out[0] = v[0];
  out[1] = v[1];
  out[3] = v[2];
  out[2] = v[4];
  out[4] = v[5];
  return BAL_OK;
}

bal_status grad_norm(Scene& S, const double* g, double* out, cudaStream_t st) {
  BAL_TRY(launch_dot(S, 3 * (int64_t)S.d.nv, g, g, 10, st));
  double v;
  BAL_TRY(read_scalars(S, &v, 10, 1, st));
  *out = std::sqrt(v);
  return BAL_OK;
}

// sigma0 (Sec. 3.4) at x with active keys A
bal_status initial_sigma(Scene& S, const double* x, const std::vector<uint64_t>& A, double* out,
                         cudaStream_t st) {
  const double floor = S.mbar / (S.d.h * S.d.h * barrier_d2b(0.5 * S.d.dhat, S.d.dhat));
  *out = floor;
  if (A.empty()) return BAL_OK;
  // grad E (inertia + elastic), then sum grad b over A with sigma = 1
  BAL_TRY(launch_inertia_elastic_grad(S, x, S.grad, st));
  std::vector<uint64_t> keep_keys = S.ap_keys;
  std::vector<double> keep_mu = S.ap_mu;
  const double keep_sigma = S.sigma;
  S.ap_keys.clear();
  S.ap_mu.clear();
  S.sigma = 1.0;
  BAL_TRY(build_eval(S, x, A, st));
  BAL_CUDA(cudaMemsetAsync(S.gtmp, 0, sizeof(double) * 3 * S.d.nv, st));
  S.fric_suspend = true;   // sigma0 weighs the barrier gradient alone
  const bal_status cs = launch_contact_terms(S, x, S.gtmp, false, st);
  S.fric_suspend = false;
  BAL_TRY(cs);
  S.ap_keys = keep_keys;
  S.ap_mu = keep_mu;
  S.sigma = keep_sigma;
  BAL_TRY(launch_dot(S, 3 * (int64_t)S.d.nv, S.gtmp, S.grad, 11, st));
  BAL_TRY(launch_dot(S, 3 * (int64_t)S.d.nv, S.gtmp, S.gtmp, 12, st));
  double v[2];
  BAL_TRY(read_scalars(S, v, 11, 2, st));
  if (v[1] > 0.0) *out = std::max(-v[0] / v[1], floor);
  return BAL_OK;
}

bal_status check_scene(const bal_scene* s) {
  if (!s) {
    set_error("null scene");
    return BAL_ERR_ARG;
  }
  return BAL_OK;
}

// One Algorithm 1 iteration on x (device, in place).
bal_status newton_iteration(Scene& S, double* x, bal_newton_info* info, cudaStream_t st) {
  const auto t_all = clk::now();
  bal_newton_info I;
  std::memset(&I, 0, sizeof(I));
  I.l = S.l;
  const double dh = S.d.dhat;
  const double thr = S.prm.ap_ratio * dh;
  const int64_t n3 = 3 * (int64_t)S.d.nv;

  auto t0 = clk::now();
  std::vector<uint64_t> A;
  std::vector<double> Ad;
  BAL_TRY(detect_active(S, x, A, Ad, st));
  double dmin = INFINITY;
  for (double d : Ad) dmin = std::min(dmin, d);
  if (S.sigma0_pending && !A.empty()) {
    // sigma0 (Sec. 3.4) needs A != empty: taken at the first iterate with contact
    double s0 = 0.0;
    BAL_TRY(initial_sigma(S, x, A, &s0, st));
    S.sigma0 = s0;
    S.sigma = s0;
    S.sigma0_pending = false;
  }
  const bool plain = S.prm.al_mode == BAL_AL_PLAIN;   // ablation: barrier only, sigma = sigma0
  if (S.l > 0 && !S.prm.freeze_al && !plain) {
    // dual update of the previous iteration, evaluated at x^[l] (Alg. 1 lines 12-15)
    if (!S.ap_keys.empty()) {
      BAL_TRY(upload_ap(S, st));
      BAL_TRY(launch_dual_update(S, x, (int64_t)S.ap_keys.size(), st));
      BAL_CUDA(cudaMemcpyAsync(S.ap_mu.data(), S.ap_mu_d.p, sizeof(double) * S.ap_mu.size(),
                               cudaMemcpyDeviceToHost, st));
      BAL_CUDA(cudaStreamSynchronize(st));
    }
    if (dmin < thr) {   // Alg. 1 line 16
      if (S.prm.sigma_literal_max)
        S.sigma = std::max(S.prm.sigma_growth * S.sigma, S.prm.sigma_cap * S.sigma0);
      else
        S.sigma = std::min(S.prm.sigma_growth * S.sigma, S.prm.sigma_cap * S.sigma0);
    }
  }
  // augmentation set rule (Alg. 1 lines 3-6); mu kept for pairs staying in A'
  if (plain) {
    S.ap_keys.clear();
    S.ap_mu.clear();
  } else if (S.prm.freeze_al) {
    // A', mu and sigma held fixed
  } else if (dmin > thr) {
    S.ap_keys.clear();
    S.ap_mu.clear();
  } else if (dmin < S.dmin_prev || S.ap_keys.empty()) {
    std::vector<uint64_t> nk;
    std::vector<double> nm;
    for (size_t i = 0; i < A.size(); ++i) {
      if (!(Ad[i] < thr)) continue;
      nk.push_back(A[i]);
      auto it = std::lower_bound(S.ap_keys.begin(), S.ap_keys.end(), A[i]);
      nm.push_back((it != S.ap_keys.end() && *it == A[i]) ? S.ap_mu[it - S.ap_keys.begin()] : 0.0);
    }
    S.ap_keys.swap(nk);
    S.ap_mu.swap(nm);
  }
  S.dmin_prev = dmin;
  BAL_TRY(build_eval(S, x, A, st));
  I.n_active = (int64_t)A.size();
  I.n_ap = (int64_t)S.ap_keys.size();
  I.dmin = dmin;
  I.sigma = S.sigma;
  I.ms_contact += ms_since(t0);

  // gradient and convergence test (Alg. 1 lines 7, 9)
  t0 = clk::now();
  BAL_TRY(gradient(S, x, S.grad, st));
  double en = 0.0;
  BAL_TRY(grad_norm(S, S.grad, &en, st));
  I.grad_norm = en;
  if (!std::isfinite(en)) {
    set_error("non-finite gradient at Newton iteration %d", S.l);
    return BAL_ERR_NAN;
  }
  if (S.l == 0) S.e0 = en;
  if (en <= S.prm.newton_abs_tol || (S.l > 0 && en <= S.prm.newton_tol * S.e0)) {
    I.converged = 1;
    if (info) *info = I;
    return BAL_OK;
  }
  BAL_TRY(assemble(S, x, nullptr, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  I.ms_assemble = ms_since(t0);

  // search direction: H p = -e
  t0 = clk::now();
  BAL_CUDA(cudaMemsetAsync(S.gtmp, 0, sizeof(double) * n3, st));
  BAL_TRY(launch_axpy(S, n3, -1.0, S.grad, S.gtmp, S.gtmp, st));   // gtmp = -grad
  BAL_CUDA(cudaMemsetAsync(S.dir, 0, sizeof(double) * n3, st));
  bal_solve_info si;
  // per-solve tolerance relative to ||r0|| = ||e|| (x0 = 0): fixed, or App. B
  // criteria (i) min(0.5, sqrt(||e||)), (ii) u kappa ||x_k|| / ||e||, (iii) u kappa
  double tol = S.prm.pcg_tol;
  if (S.prm.pcg_tol_mode == BAL_PCG_TOL_TRUNCATED_NEWTON) {
    tol = std::min(0.5, std::sqrt(en));
  } else if (S.prm.pcg_tol_mode == BAL_PCG_TOL_COND_X || S.prm.pcg_tol_mode == BAL_PCG_TOL_COND_B) {
    BAL_TRY(launch_lambda_range(S, 20, st));
    double lr[2];
    BAL_TRY(read_scalars(S, lr, 20, 2, st));
    I.kappa = lr[1] > 0.0 ? lr[0] / lr[1] : INFINITY;
    const double u = DBL_EPSILON;
    if (S.prm.pcg_tol_mode == BAL_PCG_TOL_COND_B) {
      tol = u * I.kappa;
    } else {
      BAL_TRY(launch_dot(S, n3, x, x, 22, st));
      double xx;
      BAL_TRY(read_scalars(S, &xx, 22, 1, st));
      tol = u * I.kappa * std::sqrt(xx) / en;
    }
    tol = std::min(tol, 0.5);
  }
  I.pcg_tol = tol;
  BAL_TRY(pcg_solve(S, S.gtmp, S.dir, tol, S.prm.pcg_max_iter, &si, st));
  I.pcg_iters = si.iters;
  I.pcg_rel_residual = si.rel_residual;
  I.ms_solve = ms_since(t0);

  // line search (Alg. 1 line 8; Sec. 5.2 memory cap; App. B small steps)
  t0 = clk::now();
  int extra_rounds = 0;
  for (;;) {
    auto tb = clk::now();
    BAL_TRY(find_candidates_motion(S, x, S.dir, S.ls_cand, S.ls_cand_alt, &S.n_ls_cand, st));
    I.n_raw_candidates = S.n_ls_cand;
    if (S.n_ls_cand > 0) {   // keep the pairs that can enter A or bound alpha
      BAL_TRY(buf_reserve(S.flags, S.n_ls_cand));
      BAL_TRY(buf_reserve(S.ls_cand_alt, sizeof(uint64_t) * S.n_ls_cand));
      BAL_TRY(launch_ls_filter(S, x, S.dir, S.ls_cand.as<uint64_t>(), S.n_ls_cand,
                               S.flags.as<uint8_t>(), st));
      int64_t nk = 0;
      BAL_TRY(compact_u64(S, S.ls_cand.as<uint64_t>(), S.flags.as<uint8_t>(), S.n_ls_cand,
                          S.ls_cand_alt.as<uint64_t>(), &nk, st));
      std::swap(S.ls_cand, S.ls_cand_alt);
      S.n_ls_cand = nk;
    }
    I.n_candidates = S.n_ls_cand;
    BAL_CUDA(cudaStreamSynchronize(st));
    I.ms_ls_broad += ms_since(tb);
    tb = clk::now();
    double alpha = 1.0;
    if (S.n_ls_cand > 0) {
      if (S.prm.step_mode == BAL_STEP_CCD)
        BAL_TRY(launch_ccd_bound(S, x, S.dir, S.ls_cand.as<uint64_t>(), S.n_ls_cand, 14, st));
      else
        BAL_TRY(launch_step_bound(S, x, S.dir, S.ls_cand.as<uint64_t>(), S.n_ls_cand, 14, st));
      double ab;
      BAL_TRY(read_scalars(S, &ab, 14, 1, st));
      alpha = std::min(1.0, ab);
    }
    I.ms_ls_bound += ms_since(tb);
    tb = clk::now();
    double P0[5];
    BAL_TRY(energy_parts(S, x, S.ls_cand.as<uint64_t>(), S.n_ls_cand, P0, st));
    const double E_old = P0[0] + P0[1] + P0[2];
    const double slack = S.prm.ls_slack * (std::fabs(P0[0]) + std::fabs(P0[1]) + std::fabs(P0[2]));
    int trials = 0;
    bool ok = false;
    while (alpha >= S.prm.ls_min_alpha) {
      ++trials;
      BAL_TRY(launch_axpy(S, n3, alpha, S.dir, x, S.xtrial, st));
      double P1[5];
      BAL_TRY(energy_parts(S, S.xtrial, S.ls_cand.as<uint64_t>(), S.n_ls_cand, P1, st));
      if (P1[3] > 0.0 || P1[4] > (double)S.prm.contact_cap) {
        alpha *= 0.5;
        continue;
      }
      const double E_new = P1[0] + P1[1] + P1[2];
      if (E_new - E_old <= slack) {
        ok = true;
        I.energy = E_new;
        break;
      }
      alpha *= 0.5;
    }
    I.ls_trials += trials;
    I.ms_ls_energy += ms_since(tb);
    if (ok) {
      I.alpha = alpha;
      BAL_CUDA(cudaMemcpyAsync(x, S.xtrial, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
      break;
    }
    if (extra_rounds < S.prm.ls_extra_rounds && S.prm.ls_extra_pcg > 0) {
      // App. B: step below alpha_min -> more PCG iterations on the same system,
      // continuing from the current direction, until the step grows
      ++extra_rounds;
      BAL_TRY(pcg_solve(S, S.gtmp, S.dir, 0.0, S.prm.ls_extra_pcg, &si, st));
      I.pcg_iters += si.iters;
      continue;
    }
    I.ms_line_search = ms_since(t0);
    if (info) *info = I;
    S.l += 1;
    set_error("line search: step length below %g at Newton iteration %d", S.prm.ls_min_alpha, I.l);
    return BAL_ERR_LINE_SEARCH;
  }
  I.ms_line_search = ms_since(t0);
  S.l += 1;
  (void)t_all;
  if (info) *info = I;
  return BAL_OK;
}

// a = dL/dx_{t+1} + dL/dv_{t+1} / h on free vertices, 0 on pinned ones
__global__ void k_adj_rhs(Dev S, const double* __restrict__ gx, const double* __restrict__ gv,
                          double* __restrict__ a) {
  const double ih = 1.0 / S.h;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x)
    st3(a, v, S.pinned[v] ? d3{0, 0, 0} : ld3(gx, v) + ih * ld3(gv, v));
}
// dL/dx_t = M lam / h^2 - dL/dv_{t+1} / h, dL/dv_t = M lam / h on free vertices
__global__ void k_adj_out(Dev S, const double* __restrict__ lam, const double* __restrict__ gv,
                          double* __restrict__ dx, double* __restrict__ dv) {
  const double ih = 1.0 / S.h;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < S.nv; v += gridDim.x * blockDim.x) {
    if (S.pinned[v]) {
      st3(dx, v, d3{0, 0, 0});
      st3(dv, v, d3{0, 0, 0});
      continue;
    }
    const d3 ml = S.mass[v] * ld3(lam, v);
    st3(dx, v, (ih * ih) * ml - ih * ld3(gv, v));
    st3(dv, v, ih * ml);
  }
}

__global__ void k_velocity(int64_t n, double ih, const double* __restrict__ x,
                           const double* __restrict__ xt, double* __restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (x[i] - xt[i]) * ih;
}

}  // namespace
}  // namespace bal

using namespace bal;

extern "C" {

const char* bal_last_error(void) { return g_err; }

uint64_t bal_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t bal_struct_size(int32_t which) {
  switch (which) {
    case 0: return sizeof(bal_params);
    case 1: return sizeof(bal_scene_desc);
    case 2: return sizeof(bal_bsr_view);
    case 3: return sizeof(bal_al_state);
    case 4: return sizeof(bal_solve_info);
    case 5: return sizeof(bal_newton_info);
    case 6: return sizeof(bal_step_info);
    default: return 0;
  }
}

static bool params_ok(const bal_params* p) {
  return p && !(!(p->pcg_tol >= 0) || p->pcg_max_iter < 0 || p->newton_max_iter < 0 ||
      p->precision < BAL_PREC_FP64 || p->precision > BAL_PREC_FP32 ||
      p->precond < BAL_PRECOND_BJ || p->precond > BAL_PRECOND_ADDITIVE ||
      p->step_mode < BAL_STEP_CA || p->step_mode > BAL_STEP_CCD ||
      p->broad_phase < BAL_BROAD_GRID || p->broad_phase > BAL_BROAD_LBVH ||
      p->al_mode < BAL_AL_ALGORITHM1 || p->al_mode > BAL_AL_PLAIN ||
      p->pcg_tol_mode < BAL_PCG_TOL_FIXED || p->pcg_tol_mode > BAL_PCG_TOL_COND_B ||
      !(p->step_bound > 0 && p->step_bound < 1) || !(p->sigma_growth >= 1) ||
      !(p->friction >= 0) || !(p->friction_eps_v >= 0) ||
      p->spmv_window < 0 || p->spmv_window > 4096 || (p->spmv_window % 32) != 0 ||
      p->ls_extra_rounds < 0 || !(p->pcg_stall_forcing >= 0) ||
      p->mixed_operator < BAL_MIXED_OP_DIFFERENCE || p->mixed_operator > BAL_MIXED_OP_PLAIN);
}

void bal_default_params(bal_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->precision = BAL_PREC_FP64;
  p->precond = BAL_PRECOND_BJ;
  p->pcg_tol = 1e-4;
  p->pcg_max_iter = 10000;
  p->pcg_stall_window = 100;
  p->newton_tol = 1e-4;
  p->newton_abs_tol = 0.0;
  p->newton_max_iter = 200;
  p->ap_ratio = 1e-2;
  p->sigma_growth = 1.2;
  p->sigma_cap = 100.0;
  p->sigma_literal_max = 1;
  p->step_bound = 0.9;
  p->ls_min_alpha = 1e-9;
  p->ls_slack = 1e-12;
  p->contact_cap = (int64_t)1 << 40;
  p->ls_extra_pcg = 100;
  p->warm_tol = 1e-2;
  p->warm_max_iter = 50;
  p->mixed_inner_max = 3000;
  p->mixed_inner_tol = 1e-2;
  p->mixed_max_refine = 40;
  p->ca_max_iter = 64;
  p->freeze_al = 0;
  p->step_mode = BAL_STEP_CA;
  p->broad_phase = BAL_BROAD_GRID;
  p->al_mode = BAL_AL_ALGORITHM1;
  p->pcg_tol_mode = BAL_PCG_TOL_FIXED;
  p->friction = 0.0;
  p->friction_eps_v = 0.0;
  p->spmv_window = 0;
  p->ls_extra_rounds = 10;
  p->pcg_stall_forcing = 0.0;
  p->mixed_operator = BAL_MIXED_OP_DIFFERENCE;
}

bal_status bal_create_scene(const bal_scene_desc* desc, const bal_params* params, bal_scene** out) {
  if (!desc || !out) {
    set_error("bal_create_scene: null argument");
    return BAL_ERR_ARG;
  }
  *out = nullptr;
  if (desc->n_verts <= 0 || desc->n_tets < 0 || desc->n_tris < 0 || desc->n_edges < 0 ||
      desc->n_surf_verts < 0 || !desc->X || (desc->n_tets > 0 && !desc->tets) ||
      !(desc->h > 0) || !(desc->dhat > 0) || !desc->E || !desc->nu || !desc->rho ||
      !desc->pinned || (desc->n_tris > 0 && !desc->tris) || (desc->n_edges > 0 && !desc->edges) ||
      (desc->n_surf_verts > 0 && !desc->surf_verts)) {
    set_error("bal_create_scene: invalid sizes, pointers, h or dhat");
    return BAL_ERR_ARG;
  }
  const int nv = desc->n_verts, nt = desc->n_tets;
  for (int64_t i = 0; i < 4 * (int64_t)nt; ++i)
    if (desc->tets[i] < 0 || desc->tets[i] >= nv) {
      set_error("bal_create_scene: tet vertex index out of range at %lld", (long long)i);
      return BAL_ERR_ARG;
    }
  for (int64_t i = 0; i < 3 * (int64_t)desc->n_tris; ++i)
    if (desc->tris[i] < 0 || desc->tris[i] >= nv) {
      set_error("bal_create_scene: triangle vertex index out of range");
      return BAL_ERR_ARG;
    }
  for (int64_t i = 0; i < 2 * (int64_t)desc->n_edges; ++i)
    if (desc->edges[i] < 0 || desc->edges[i] >= nv) {
      set_error("bal_create_scene: edge vertex index out of range");
      return BAL_ERR_ARG;
    }
  for (int64_t i = 0; i < desc->n_surf_verts; ++i)
    if (desc->surf_verts[i] < 0 || desc->surf_verts[i] >= nv) {
      set_error("bal_create_scene: surface vertex index out of range");
      return BAL_ERR_ARG;
    }
  if (params && !params_ok(params)) {
    set_error("bal_create_scene: invalid parameters");
    return BAL_ERR_ARG;
  }
  bal_scene* sc = new bal_scene();
  Scene& S = sc->S;
  S.d.nv = nv;
  S.d.nt = nt;
  S.d.nf = desc->n_tris;
  S.d.ne = desc->n_edges;
  S.d.nsv = desc->n_surf_verts;
  S.d.h = desc->h;
  S.d.dhat = desc->dhat;
  for (int k = 0; k < 3; ++k) S.grav[k] = desc->gravity[k];
  if (params) S.prm = *params; else bal_default_params(&S.prm);
  S.pair_limit = desc->pair_limit > 0 ? desc->pair_limit : ((int64_t)1 << 31) - 1;

  // rest data (Sec. 3.1): D_m^{-1}, V_e, Lame parameters, lumped mass
  std::vector<double> Dmi(9 * (size_t)nt), vol(nt), mu(nt), lam(nt), mass(nv, 0.0);
  const double* X = desc->X;
  for (int t = 0; t < nt; ++t) {
    const int* v = desc->tets + 4 * (int64_t)t;
    double M[3][3];
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 3; ++i) M[i][a] = X[3 * v[a + 1] + i] - X[3 * v[0] + i];
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(std::fabs(det) > 0.0)) {
      delete sc;
      set_error("bal_create_scene: degenerate rest tet %d", t);
      return BAL_ERR_ARG;
    }
    double* o = Dmi.data() + 9 * (size_t)t;
    o[0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
    o[1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
    o[2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
    o[3] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
    o[4] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
    o[5] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
    o[6] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
    o[7] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
    o[8] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
    vol[t] = std::fabs(det) / 6.0;
    const double E = desc->E[t], nu = desc->nu[t];
    mu[t] = E / (2.0 * (1.0 + nu));
    lam[t] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double share = desc->rho[t] * vol[t] / 4.0;
    for (int a = 0; a < 4; ++a) mass[v[a]] += share;
  }
  double msum = 0.0;
  for (double m : mass) msum += m;
  S.mbar = msum / nv;
  S.mass_h = mass;

  // static lower pattern from node adjacency (Sec. 5.1, App. C) + tet -> slot map
  std::vector<uint64_t> pk;
  pk.reserve(6 * (size_t)nt);
  static const int pa[6] = {1, 2, 3, 2, 3, 3}, pb[6] = {0, 0, 0, 1, 1, 2};
  for (int t = 0; t < nt; ++t) {
    const int* v = desc->tets + 4 * (int64_t)t;
    for (int k = 0; k < 6; ++k) {
      const uint32_t a = (uint32_t)v[pa[k]], b = (uint32_t)v[pb[k]];
      const uint32_t r = a > b ? a : b, c = a > b ? b : a;
      pk.push_back(((uint64_t)r << 32) | c);
    }
  }
  std::vector<uint64_t> uk = pk;
  std::sort(uk.begin(), uk.end());
  uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
  S.d.nnzL = (int64_t)uk.size();
  S.row_ptr_h.assign(nv + 1, 0);
  S.col_h.resize(uk.size());
  std::vector<int32_t> rows(uk.size());
  for (size_t i = 0; i < uk.size(); ++i) {
    rows[i] = (int32_t)(uk[i] >> 32);
    S.col_h[i] = (int32_t)(uk[i] & 0xffffffffu);
    S.row_ptr_h[rows[i] + 1]++;
  }
  for (int i = 0; i < nv; ++i) S.row_ptr_h[i + 1] += S.row_ptr_h[i];
  std::vector<int32_t> slot(6 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    const int* v = desc->tets + 4 * (int64_t)t;
    for (int k = 0; k < 6; ++k) {
      const uint64_t key = pk[6 * (size_t)t + k];
      const int64_t s = std::lower_bound(uk.begin(), uk.end(), key) - uk.begin();
      const bool transpose = v[pa[k]] < v[pb[k]];
      slot[6 * (size_t)t + k] = (int32_t)(2 * s + (transpose ? 1 : 0));
    }
  }
  // bodies: connected components of the tet mesh (union-find)
  std::vector<int32_t> parent(nv);
  for (int i = 0; i < nv; ++i) parent[i] = i;
  auto find = [&](int a) {
    while (parent[a] != a) {
      parent[a] = parent[parent[a]];
      a = parent[a];
    }
    return a;
  };
  for (int t = 0; t < nt; ++t) {
    const int* v = desc->tets + 4 * (int64_t)t;
    for (int k = 1; k < 4; ++k) {
      const int a = find(v[0]), b = find(v[k]);
      if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
  }
  std::vector<int32_t> body(nv), root_id(nv, -1);
  std::vector<double> bcnt;
  for (int i = 0; i < nv; ++i) {
    const int r = find(i);
    if (root_id[r] < 0) {
      root_id[r] = (int32_t)bcnt.size();
      bcnt.push_back(0.0);
    }
    body[i] = root_id[r];
    bcnt[body[i]] += 1.0;
  }
  for (double& c : bcnt) c = 1.0 / c;
  S.nbody = (int32_t)bcnt.size();
  // mean surface edge length at rest (grid cell size)
  // and the rest squared length of every surface edge (edge-edge mollifier)
  double el = 0.0;
  std::vector<double> edge_l2(desc->n_edges);
  for (int e = 0; e < desc->n_edges; ++e) {
    const int a = desc->edges[2 * e], b = desc->edges[2 * e + 1];
    double s2 = 0;
    for (int i = 0; i < 3; ++i) s2 += (X[3 * a + i] - X[3 * b + i]) * (X[3 * a + i] - X[3 * b + i]);
    edge_l2[e] = s2;
    el += std::sqrt(s2);
  }
  S.mean_edge = desc->n_edges ? el / desc->n_edges : 1e-3;

  bal_status st = BAL_OK;
#define TRYC(x)                 \
  do {                          \
    st = (x);                   \
    if (st != BAL_OK) goto fail; \
  } while (0)
  TRYC(dupload(S, &S.d.tets, desc->tets, 4 * (size_t)nt));
  TRYC(dupload(S, &S.d.tris, desc->tris, 3 * (size_t)desc->n_tris));
  TRYC(dupload(S, &S.d.edges, desc->edges, 2 * (size_t)desc->n_edges));
  TRYC(dupload(S, &S.d.edge_l2, (const double*)edge_l2.data(), edge_l2.size()));
  TRYC(dupload(S, &S.d.surf, desc->surf_verts, (size_t)desc->n_surf_verts));
  TRYC(dupload(S, &S.d.pinned, desc->pinned, (size_t)nv));
  TRYC(dupload(S, &S.d.Dm_inv, (const double*)Dmi.data(), Dmi.size()));
  TRYC(dupload(S, &S.d.vol, (const double*)vol.data(), vol.size()));
  TRYC(dupload(S, &S.d.mu, (const double*)mu.data(), mu.size()));
  S.E_h.assign(desc->E, desc->E + nt);
  S.nu_h.assign(desc->nu, desc->nu + nt);
  TRYC(dupload(S, (const double**)&S.E, (const double*)S.E_h.data(), S.E_h.size()));
  TRYC(dupload(S, &S.d.lam, (const double*)lam.data(), lam.size()));
  TRYC(dupload(S, &S.d.mass, (const double*)mass.data(), mass.size()));
  TRYC(dupload(S, &S.d.L_row_ptr, (const int32_t*)S.row_ptr_h.data(), S.row_ptr_h.size()));
  TRYC(dupload(S, &S.d.L_col, (const int32_t*)S.col_h.data(), S.col_h.size()));
  TRYC(dupload(S, &S.d.L_row, (const int32_t*)rows.data(), rows.size()));
  TRYC(dupload(S, &S.d.tet_slot, (const int32_t*)slot.data(), slot.size()));
  TRYC(dupload(S, (const int32_t**)&S.body, (const int32_t*)body.data(), body.size()));
  TRYC(dupload(S, (const double**)&S.body_inv_cnt, (const double*)bcnt.data(), bcnt.size()));
  TRYC(dalloc(S, &S.bmean, 3 * (size_t)S.nbody));
  TRYC(dalloc(S, &S.bmot, (size_t)S.nbody));
  TRYC(dalloc(S, &S.d.D, 9 * (size_t)nv));
  TRYC(dalloc(S, &S.d.Dinv, 9 * (size_t)nv));
  TRYC(dalloc(S, &S.d.Lval, 9 * (size_t)S.d.nnzL));
  TRYC(dalloc(S, &S.d.Lambda, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.d.y, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.xt, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.grad, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.gtmp, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.xtrial, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.dir, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pcg_r, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pcg_z, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pcg_p, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pcg_q, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pcg_x, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.pnorm, (size_t)nv));
  TRYC(dalloc(S, &S.group, (size_t)nv));
  TRYC(dalloc(S, &S.D32, 9 * (size_t)nv));
  TRYC(dalloc(S, &S.Dinv32, 9 * (size_t)nv));
  TRYC(dalloc(S, &S.Lval32, 9 * (size_t)S.d.nnzL));
  TRYC(dalloc(S, &S.b32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.x32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.r32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.z32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.p32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.q32, 3 * (size_t)nv));
  TRYC(dalloc(S, &S.partials, (size_t)kMaxPartials));
  TRYC(dalloc(S, &S.scal, 64));
  TRYC(dalloc(S, &S.pcg, 1));
  if (desc->pair_capacity > 0) TRYC(buf_reserve(S.cand, sizeof(uint64_t) * desc->pair_capacity));
  {
    cudaError_t e = cudaMemset(S.scal, 0, sizeof(double) * 64);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
      goto fail;
    }
    e = cudaMemset(S.pcg, 0, sizeof(PcgScalars));
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
      goto fail;
    }
  }
#undef TRYC
  *out = sc;
  return BAL_OK;
fail:
  bal_destroy_scene(sc);
  return st;
}

bal_status bal_destroy_scene(bal_scene* sc) {
  if (!sc) return BAL_OK;
  Scene& S = sc->S;
  for (void* p : S.owned) cudaFree(p);
  for (cudaEvent_t& e : S.kev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t& e : S.kaev)
    if (e) cudaEventDestroy(e);
  Buf* bufs[] = {&S.C_row, &S.C_col, &S.C_val, &S.C_val32, &S.f32_S, &S.emit_keys, &S.emit_vals, &S.cm_cnt,
                 &S.cm_off, &S.cm_bucket, &S.cm_sorted, &S.cm_ucnt, &S.cm_uoff, &S.scan_aux, &S.cub_tmp, &S.bp_cells,
                 &S.bp_cells_alt, &S.bp_ids, &S.bp_ids_alt, &S.bp_count, &S.bp_offs, &S.cand,
                 &S.cand_alt, &S.dist, &S.dist_alt, &S.flags, &S.eval_keys, &S.eval_flags, &S.eval_mu, &S.eval_s,
                 &S.ls_cand, &S.ls_cand_alt, &S.bstats, &S.ap_keys_d, &S.ap_mu_d, &S.ap_s_d,
                 &S.lb_pbox, &S.lb_nbox, &S.lb_keys, &S.lb_keys_alt, &S.lb_child, &S.lb_parent,
                 &S.lb_prim, &S.lb_arrivals, &S.lb_bounds, &S.add_inv,
                 &S.sell_offR, &S.sell_offT, &S.sell_Rcol, &S.sell_Tpos, &S.sell_Tsrc, &S.sell_pos, &S.sell_len,
                 &S.sell_srow, &S.sell_slot, &S.fr_keys, &S.fr_beta, &S.fr_n, &S.fr_lam,
                 &S.dd_D, &S.dd_Dinv, &S.dd_R, &S.dd_C, &S.dd_vec, &S.cr_rows, &S.cr_ptr, &S.cr_ent,
                 &S.cr_src, &S.cr_key, &S.cr_bucket, &S.cr_sorted, &S.cr_cnt, &S.cr_off, &S.cr_len, &S.cr_rpos,
                 &S.cr_of, &S.cr_q};
  for (Buf* b : bufs) buf_free(*b);
  delete sc;
  return BAL_OK;
}

bal_status bal_set_params(bal_scene* sc, const bal_params* p) {
  BAL_TRY(check_scene(sc));
  if (!params_ok(p)) {
    set_error("bal_set_params: invalid parameters");
    return BAL_ERR_ARG;
  }
  sc->S.prm = *p;
  return BAL_OK;
}

bal_status bal_kernel_timing(bal_scene* sc, int32_t enable, double* total_ms, int64_t* launches) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (total_ms) *total_ms = S.kt_ms;
  if (launches) *launches = S.kt_n;
  S.kt_ms = 0;
  S.kt_n = 0;
  if (enable && !S.kev[0]) {
    for (cudaEvent_t& e : S.kev) BAL_CUDA(cudaEventCreate(&e));
    for (cudaEvent_t& e : S.kaev) BAL_CUDA(cudaEventCreate(&e));
  }
  S.ktime = enable != 0;
  return BAL_OK;
}

bal_status bal_assembly_timing(bal_scene* sc, double* elastic_ms, double* total_ms, int64_t* assemblies) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (elastic_ms) *elastic_ms = S.ka_elastic_ms;
  if (total_ms) *total_ms = S.ka_total_ms;
  if (assemblies) *assemblies = S.ka_n;
  S.ka_elastic_ms = S.ka_total_ms = 0;
  S.ka_n = 0;
  return BAL_OK;
}

bal_status bal_get_params(const bal_scene* sc, bal_params* out) {
  BAL_TRY(check_scene(sc));
  if (!out) return BAL_ERR_ARG;
  *out = sc->S.prm;
  return BAL_OK;
}

bal_status bal_static_pattern(const bal_scene* sc, int64_t* nnz, int32_t* row_ptr, int32_t* col) {
  BAL_TRY(check_scene(sc));
  const Scene& S = sc->S;
  if (nnz) *nnz = S.d.nnzL;
  if (row_ptr) std::memcpy(row_ptr, S.row_ptr_h.data(), sizeof(int32_t) * S.row_ptr_h.size());
  if (col) std::memcpy(col, S.col_h.data(), sizeof(int32_t) * S.col_h.size());
  return BAL_OK;
}

bal_status bal_get_mass(const bal_scene* sc, double* m) {
  BAL_TRY(check_scene(sc));
  if (!m) return BAL_ERR_ARG;
  std::memcpy(m, sc->S.mass_h.data(), sizeof(double) * sc->S.mass_h.size());
  return BAL_OK;
}

bal_status bal_step_begin(bal_scene* sc, const double* x_t, const double* v_t, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!x_t || !v_t) {
    set_error("bal_step_begin: null x_t or v_t");
    return BAL_ERR_ARG;
  }
  Scene& S = sc->S;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  BAL_CUDA(cudaMemcpyAsync(S.xt, x_t, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
  BAL_TRY(launch_make_y(S, x_t, v_t, S.d.y, st));
  S.dmin_prev = INFINITY;
  S.l = 0;
  S.e0 = 0.0;
  S.n_fr = 0;
  S.step_active = true;
  S.sigma0_pending = false;
  if (S.prm.freeze_al) return BAL_OK;   // keep sigma, A', mu as set by bal_set_al_state
  S.ap_keys.clear();
  S.ap_mu.clear();
  std::vector<uint64_t> A;
  std::vector<double> Ad;
  BAL_TRY(detect_active(S, x_t, A, Ad, st));
  S.sigma = 1.0;
  double s0 = 0.0;
  BAL_TRY(initial_sigma(S, x_t, A, &s0, st));
  S.sigma0 = s0;
  S.sigma = s0;
  S.sigma0_pending = A.empty();
  return BAL_OK;
}

bal_status bal_get_al_state(const bal_scene* sc, bal_al_state* out, int64_t capacity) {
  BAL_TRY(check_scene(sc));
  if (!out) return BAL_ERR_ARG;
  const Scene& S = sc->S;
  out->sigma = S.sigma;
  out->sigma0 = S.sigma0;
  out->dmin_prev = S.dmin_prev;
  out->n_ap = (int64_t)S.ap_keys.size();
  if (out->ap_keys && out->ap_mu) {
    if (capacity < out->n_ap) {
      set_error("bal_get_al_state: capacity %lld < |A'| %lld", (long long)capacity, (long long)out->n_ap);
      return BAL_ERR_ARG;
    }
    std::memcpy(out->ap_keys, S.ap_keys.data(), sizeof(uint64_t) * S.ap_keys.size());
    std::memcpy(out->ap_mu, S.ap_mu.data(), sizeof(double) * S.ap_mu.size());
  }
  return BAL_OK;
}

bal_status bal_set_al_state(bal_scene* sc, const bal_al_state* in) {
  BAL_TRY(check_scene(sc));
  if (!in || in->n_ap < 0 || (in->n_ap > 0 && (!in->ap_keys || !in->ap_mu)) || !(in->sigma > 0)) {
    set_error("bal_set_al_state: invalid state");
    return BAL_ERR_ARG;
  }
  Scene& S = sc->S;
  S.sigma = in->sigma;
  S.sigma0 = in->sigma0;
  S.sigma0_pending = false;
  S.dmin_prev = in->dmin_prev;
  S.ap_keys.assign(in->ap_keys, in->ap_keys + in->n_ap);
  S.ap_mu.assign(in->ap_mu, in->ap_mu + in->n_ap);
  for (int64_t i = 1; i < in->n_ap; ++i)
    if (!(S.ap_keys[i - 1] < S.ap_keys[i])) {
      set_error("bal_set_al_state: keys must be sorted ascending and unique");
      return BAL_ERR_ARG;
    }
  return BAL_OK;
}

bal_status bal_get_y(const bal_scene* sc, double* y_out, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!y_out) return BAL_ERR_ARG;
  const Scene& S = sc->S;
  BAL_CUDA(cudaMemcpyAsync(y_out, S.d.y, sizeof(double) * 3 * S.d.nv, cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  BAL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return BAL_OK;
}

bal_status bal_assemble_hessian(bal_scene* sc, const double* x, double* grad_out, bal_bsr_view* view,
                                void* stream) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (!x) return BAL_ERR_ARG;
  if (!S.step_active) {
    set_error("bal_assemble_hessian: call bal_step_begin first");
    return BAL_ERR_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint64_t> A;
  std::vector<double> Ad;
  BAL_TRY(detect_active(S, x, A, Ad, st));
  BAL_TRY(build_eval(S, x, A, st));
  BAL_TRY(launch_inertia_elastic_grad(S, x, S.grad, st));
  BAL_TRY(assemble(S, x, S.grad, st));
  if (grad_out)
    BAL_CUDA(cudaMemcpyAsync(grad_out, S.grad, sizeof(double) * 3 * S.d.nv, cudaMemcpyDeviceToDevice, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  if (view) {
    view->n_verts = S.d.nv;
    view->nnz_L = S.d.nnzL;
    view->nnz_C = S.nnzC;
    view->D = S.d.D;
    view->L_row_ptr = S.d.L_row_ptr;
    view->L_col = S.d.L_col;
    view->L_val = S.d.Lval;
    view->C_row = S.C_row.as<int32_t>();
    view->C_col = S.C_col.as<int32_t>();
    view->C_val = S.C_val.as<double>();
    view->Lambda = S.d.Lambda;
  }
  return BAL_OK;
}

bal_status bal_copy_hessian(bal_scene* sc, double* D_out, double* L_out, int32_t* Cr, int32_t* Cc,
                            double* Cv, double* Lam, void* stream) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (!S.assembled) {
    set_error("bal_copy_hessian: no assembled Hessian");
    return BAL_ERR_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const auto d2d = cudaMemcpyDeviceToDevice;
  if (D_out) BAL_CUDA(cudaMemcpyAsync(D_out, S.d.D, sizeof(double) * 9 * S.d.nv, d2d, st));
  if (L_out && S.d.nnzL) BAL_CUDA(cudaMemcpyAsync(L_out, S.d.Lval, sizeof(double) * 9 * S.d.nnzL, d2d, st));
  if (S.nnzC) {
    if (Cr) BAL_CUDA(cudaMemcpyAsync(Cr, S.C_row.p, sizeof(int32_t) * S.nnzC, d2d, st));
    if (Cc) BAL_CUDA(cudaMemcpyAsync(Cc, S.C_col.p, sizeof(int32_t) * S.nnzC, d2d, st));
    if (Cv) BAL_CUDA(cudaMemcpyAsync(Cv, S.C_val.p, sizeof(double) * 9 * S.nnzC, d2d, st));
  }
  if (Lam) BAL_CUDA(cudaMemcpyAsync(Lam, S.d.Lambda, sizeof(double) * 3 * S.d.nv, d2d, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}

bal_status bal_spmv(bal_scene* sc, const double* v, double* y, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!v || !y) return BAL_ERR_ARG;
  if (!sc->S.assembled) {
    set_error("bal_spmv: no assembled Hessian");
    return BAL_ERR_STATE;
  }
  BAL_TRY(spmv(sc->S, v, y, (cudaStream_t)stream));
  return BAL_OK;
}

bal_status bal_pcg_solve(bal_scene* sc, const double* rhs, double* sol, double rel_tol, int32_t max_iter,
                         bal_solve_info* info, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!rhs || !sol || !(rel_tol >= 0) || max_iter < 0) return BAL_ERR_ARG;
  if (!sc->S.assembled) {
    set_error("bal_pcg_solve: no assembled Hessian");
    return BAL_ERR_STATE;
  }
  bal_solve_info local;
  return pcg_solve(sc->S, rhs, sol, rel_tol, max_iter, info ? info : &local, (cudaStream_t)stream);
}

bal_status bal_energy(bal_scene* sc, const double* x, double* e, void* stream) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (!x || !e) return BAL_ERR_ARG;
  if (!S.step_active) {
    set_error("bal_energy: call bal_step_begin first");
    return BAL_ERR_STATE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint64_t> A;
  std::vector<double> Ad;
  BAL_TRY(detect_active(S, x, A, Ad, st));
  BAL_TRY(build_eval(S, x, A, st));
  if (S.prm.friction > 0.0) BAL_TRY(launch_contact_terms(S, x, nullptr, false, st));   // lag friction at x
  double P[5];
  BAL_TRY(energy_parts(S, x, S.cand.as<uint64_t>(), S.n_cand, P, st));
  *e = P[3] > 0 ? INFINITY : P[0] + P[1] + P[2];
  return BAL_OK;
}

// candidates along x + t dir: the swept LBVH query at radius r, or the grid's
// motion pass (whose radius is fixed by the line-search rule)
static bal_status lbvh_or_grid_motion(Scene& S, const double* x, const double* dir, double r, int64_t* n,
                                      cudaStream_t st) {
  if (S.prm.broad_phase == BAL_BROAD_LBVH) return lbvh_candidates(S, x, dir, r, S.cand_alt, S.ls_cand_alt, n, st);
  return find_candidates_motion(S, x, dir, S.cand_alt, S.ls_cand_alt, n, st);
}

bal_status bal_find_candidates(bal_scene* sc, const double* x, const double* dir, double r,
                               uint64_t* keys_out, int64_t capacity, int64_t* n_out, void* stream) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (!x || !n_out || !(r >= 0) || capacity < 0 || (capacity > 0 && !keys_out)) return BAL_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t n = 0;
  if (dir) BAL_TRY(lbvh_or_grid_motion(S, x, dir, r, &n, st));
  else BAL_TRY(find_candidates(S, x, r, S.cand_alt, S.ls_cand_alt, &n, st));
  *n_out = n;
  if (n > capacity) {
    set_error("bal_find_candidates: %lld pairs exceed the capacity %lld", (long long)n, (long long)capacity);
    return BAL_ERR_CAPACITY;
  }
  if (n > 0)
    BAL_CUDA(cudaMemcpyAsync(keys_out, S.cand_alt.p, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  return BAL_OK;
}

bal_status bal_step_bound(bal_scene* sc, const double* x, const double* dir, const uint64_t* pair_keys,
                          int64_t n_pairs, int32_t mode, double* alpha_out, void* stream) {
  BAL_TRY(check_scene(sc));
  Scene& S = sc->S;
  if (!x || !dir || !alpha_out || n_pairs < 0 || (n_pairs > 0 && !pair_keys) ||
      (mode != BAL_STEP_CA && mode != BAL_STEP_CCD))
    return BAL_ERR_ARG;
  *alpha_out = 1.0;
  if (n_pairs == 0) return BAL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == BAL_STEP_CCD) BAL_TRY(launch_ccd_bound(S, x, dir, pair_keys, n_pairs, 14, st));
  else BAL_TRY(launch_step_bound(S, x, dir, pair_keys, n_pairs, 14, st));
  double ab;
  BAL_TRY(read_scalars(S, &ab, 14, 1, st));
  *alpha_out = std::min(1.0, ab);
  return BAL_OK;
}

bal_status bal_newton_step(bal_scene* sc, double* x, bal_newton_info* info, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!x) return BAL_ERR_ARG;
  if (!sc->S.step_active) {
    set_error("bal_newton_step: call bal_step_begin first");
    return BAL_ERR_STATE;
  }
  return newton_iteration(sc->S, x, info, (cudaStream_t)stream);
}

bal_status bal_set_materials(bal_scene* sc, const double* E, const double* nu) {
  BAL_TRY(check_scene(sc));
  if (!E || !nu) return BAL_ERR_ARG;
  Scene& S = sc->S;
  const int nt = S.d.nt;
  std::vector<double> mu(nt), lam(nt);
  for (int t = 0; t < nt; ++t) {
    if (!(E[t] > 0) || !(nu[t] > -1 && nu[t] < 0.5)) {
      set_error("bal_set_materials: invalid E or nu at tet %d", t);
      return BAL_ERR_ARG;
    }
    mu[t] = E[t] / (2.0 * (1.0 + nu[t]));
    lam[t] = E[t] * nu[t] / ((1.0 + nu[t]) * (1.0 - 2.0 * nu[t]));
  }
  S.E_h.assign(E, E + nt);
  S.nu_h.assign(nu, nu + nt);
  BAL_CUDA(cudaMemcpy((void*)S.d.mu, mu.data(), sizeof(double) * nt, cudaMemcpyHostToDevice));
  BAL_CUDA(cudaMemcpy((void*)S.d.lam, lam.data(), sizeof(double) * nt, cudaMemcpyHostToDevice));
  BAL_CUDA(cudaMemcpy(S.E, E, sizeof(double) * nt, cudaMemcpyHostToDevice));
  return BAL_OK;
}

bal_status bal_adjoint_step(bal_scene* sc, const double* x_t, const double* v_t, const double* x_next,
                            const bal_al_state* al, const double* gx, const double* gv, double* dx,
                            double* dv, double* dE, double rel_tol, int32_t max_iter,
                            bal_solve_info* info, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!x_t || !v_t || !x_next || !al || !gx || !gv || !dx || !dv || !dE || !(rel_tol >= 0) ||
      max_iter < 0) {
    set_error("bal_adjoint_step: invalid argument");
    return BAL_ERR_ARG;
  }
  Scene& S = sc->S;
  if (S.prm.friction > 0.0) {
    set_error("bal_adjoint_step: friction > 0 is not differentiated");
    return BAL_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  BAL_TRY(launch_make_y(S, x_t, v_t, S.d.y, st));
  BAL_TRY(bal_set_al_state(sc, al));
  S.step_active = true;
  std::vector<uint64_t> A;
  std::vector<double> Ad;
  BAL_TRY(detect_active(S, x_next, A, Ad, st));
  BAL_TRY(build_eval(S, x_next, A, st));
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  k_adj_rhs<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, gx, gv, S.gtmp);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  bal_solve_info si;
  std::memset(&si, 0, sizeof(si));
  S.project = false;
  bal_status s = assemble(S, x_next, nullptr, st);
  S.project = true;
  BAL_TRY(s);
  BAL_CUDA(cudaMemsetAsync(S.dir, 0, sizeof(double) * n3, st));
  const int32_t keep_precond = S.prm.precond, keep_prec = S.prm.precision;
  S.prm.precond = BAL_PRECOND_BJ;
  S.prm.precision = BAL_PREC_FP64;
  s = pcg_solve(S, S.gtmp, S.dir, rel_tol, max_iter, &si, st);
  if (s == BAL_ERR_NAN) {   // indefinite: fall back to the projected Hessian
    BAL_TRY(assemble(S, x_next, nullptr, st));
    BAL_CUDA(cudaMemsetAsync(S.dir, 0, sizeof(double) * n3, st));
    s = pcg_solve(S, S.gtmp, S.dir, rel_tol, max_iter, &si, st);
    si.negative_curvature = 1;
  }
  S.prm.precond = keep_precond;
  S.prm.precision = keep_prec;
  BAL_TRY(s);
  k_adj_out<<<grid_for(S.d.nv), kThreads, 0, st>>>(S.d, S.dir, gv, dx, dv);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_TRY(launch_dLdE(S, x_next, S.dir, dE, st));
  BAL_CUDA(cudaStreamSynchronize(st));
  if (info) *info = si;
  return BAL_OK;
}

bal_status bal_step_end(bal_scene* sc, const double* x, double* v, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!x || !v) {
    set_error("bal_step_end: null x or v");
    return BAL_ERR_ARG;
  }
  Scene& S = sc->S;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  k_velocity<<<grid_for(n3), kThreads, 0, st>>>(n3, 1.0 / S.d.h, x, S.xt, v);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  return BAL_OK;
}

bal_status bal_time_step(bal_scene* sc, double* x, double* v, bal_step_info* info, void* stream) {
  BAL_TRY(check_scene(sc));
  if (!x || !v) return BAL_ERR_ARG;
  Scene& S = sc->S;
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = clk::now();
  bal_step_info I;
  std::memset(&I, 0, sizeof(I));
  I.min_distance = INFINITY;
  BAL_TRY(bal_step_begin(sc, x, v, stream));
  I.sigma0 = S.sigma0;
  bal_status status = BAL_ERR_NOT_CONVERGED;
  for (int l = 0; l < S.prm.newton_max_iter; ++l) {
    bal_newton_info ni;
    std::memset(&ni, 0, sizeof(ni));
    const bal_status s = newton_iteration(S, x, &ni, st);
    I.ms_assemble += ni.ms_assemble;
    I.ms_solve += ni.ms_solve;
    I.ms_line_search += ni.ms_line_search;
    I.ms_contact += ni.ms_contact;
    I.pcg_iters_total += ni.pcg_iters;
    I.max_active = std::max(I.max_active, ni.n_active);
    I.min_distance = std::min(I.min_distance, ni.dmin);
    if (s != BAL_OK) {
      status = s;
      break;
    }
    if (ni.converged) {
      status = BAL_OK;
      I.converged = 1;
      break;
    }
    I.newton_iters += 1;
  }
  I.sigma_final = S.sigma;
  I.sigma0 = S.sigma0;
  // v = (x - x_t) / h (Sec. 3.1)
  const int64_t n3 = 3 * (int64_t)S.d.nv;
  k_velocity<<<grid_for(n3), kThreads, 0, st>>>(n3, 1.0 / S.d.h, x, S.xt, v);
  ::bal::note_launch();
  BAL_LAUNCH_CHECK();
  BAL_CUDA(cudaStreamSynchronize(st));
  I.ms_total = ms_since(t0);
  if (info) *info = I;
  if (status == BAL_ERR_NOT_CONVERGED)
    set_error("bal_time_step: no convergence in %d Newton iterations", S.prm.newton_max_iter);
  return status;
}

}  // extern "C"
