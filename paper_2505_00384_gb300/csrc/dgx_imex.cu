// One IMEX step of the compressible-Euler scheme (arXiv:2505.00384, Sec. 2):
// the stage equations of an IMEX Runge-Kutta pair (A, A~) with an explicit
// first stage, the explicit sums m^(l), e^(l), and per implicit stage K
// fixed-point iterations of the pressure (Helmholtz) equation, each one
// linear solve of D P + C A^-1 (F - B P) = G (Sec. 2, fixed-point form).
//
// Stage l (rho' = rho - rho_bar, p' = p - p_bar, alpha = a~_ll dt):
//   rho^(l) = rho^n + M^-1 dt sum_m a_lm Erho^(m)
//   F = A(rho^n) u^n + dt sum_m (a_lm Em^(m) + a~_lm Im^(m)) + alpha int rho'^(l) g.phi
//   G = D p'^n + int rho^n k^n psi + dt sum_m (a_lm Ee^(m) + a~_lm Ie^(m)) - int rho^(l) k^(l,k) psi
//   solve (D - C A^-1 B) p' = G - C A^-1 F,  U = A^-1 (F - B p')
// with Erho, Em, Ee the explicit tendencies (continuity, momentum advection,
// kinetic-energy flux + gravity work) and Im = -B_1 p' + int rho' g.phi,
// Ie = -C_1 u the implicit-type terms of earlier stages.  The tableau must be
// stiffly accurate: the new state is the last stage.
#include <chrono>
#include <cmath>
#include <cstring>

#include "dgx_common.cuh"

using namespace dgx;

namespace {

struct ImexWS {
  double *Ten;  // 9N per stage: Erho, Em(3), Ee, Im(3), Ie
  double *rn, *un, *pn, *rl, *ul, *pl, *Fs, *Gs, *W, *rhs, *x, *t1, *t2, *zeros, *ones;
};

int imex_workspace(dgx_ctx *c, ImexWS &w) {
  const size_t N = (size_t)c->N;
  const size_t need = 9 * N * c->imex_s + 27 * N;
  if (c->imex_ws_elems < need) {
    if (c->imex_ws) cudaFree(c->imex_ws);
    c->imex_ws = nullptr;
    c->imex_ws_elems = 0;
    if (int e = check_cuda(c, cudaMalloc(&c->imex_ws, need * sizeof(double)), "cudaMalloc IMEX workspace")) return e;
    c->imex_ws_elems = need;
  }
  double *q = c->imex_ws;
  w.Ten = q;
  q += 9 * N * c->imex_s;
  auto take = [&](size_t n) {
    double *r = q;
    q += n;
    return r;
  };
  w.rn = take(N); w.un = take(3 * N); w.pn = take(N);
  w.rl = take(N); w.ul = take(3 * N); w.pl = take(N);
  w.Fs = take(3 * N); w.Gs = take(N); w.W = take(3 * N); w.rhs = take(N); w.x = take(N);
  w.t1 = take(3 * N); w.t2 = take(3 * N); w.zeros = take(N); w.ones = take(N);
  return 0;
}

__global__ void k_fill(long long n, double v, double *__restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

int grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 608 ? (b < 1 ? 1 : b) : 608);
}

int ready(dgx_ctx *c) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_mesh) return set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (!c->has_bg) return set_error(c, DGX_ERR_STATE, "no background (call dgx_set_background)");
  return 0;
}

}  // namespace

extern "C" {

int dgx_set_imex(dgx_ctx *c, int s, const double *A, const double *At, double dt, int K) {
  if (!c) return DGX_ERR_ARG;
  if (s < 2 || s > 4 || !A || !At) return set_error(c, DGX_ERR_ARG, "need 2 <= s <= 4 stages and both tableaux");
  if (!(dt > 0) || K < 1 || K > 50) return set_error(c, DGX_ERR_ARG, "need dt > 0 and 1 <= K <= 50");
  for (int l = 0; l < s; ++l)
    for (int m = 0; m < s; ++m) {
      if (m >= l && A[l * s + m] != 0.0) return set_error(c, DGX_ERR_ARG, "explicit tableau must be strictly lower");
      if (m > l && At[l * s + m] != 0.0) return set_error(c, DGX_ERR_ARG, "implicit tableau must be lower triangular");
    }
  for (int m = 0; m < s; ++m)
    if (At[m] != 0.0) return set_error(c, DGX_ERR_ARG, "the first stage must be explicit (a~_1m = 0)");
  for (int l = 1; l < s; ++l)
    if (!(At[l * s + l] > 0.0)) return set_error(c, DGX_ERR_ARG, "stages after the first need a~_ll > 0");
  c->imex_s = s;
  std::memcpy(c->imex_A, A, sizeof(double) * s * s);
  std::memcpy(c->imex_At, At, sizeof(double) * s * s);
  c->imex_dt = dt;
  c->imex_K = K;
  c->has_imex = true;
  return DGX_OK;
}

int dgx_explicit_tendencies(dgx_ctx *c, const double *rho, const double *u, double *Erho, double *Em, double *Ee) {
  if (int e = ready(c)) return e;
  if (!rho || !u || !Erho || !Em || !Ee) return set_error(c, DGX_ERR_ARG, "null array");
  return launch_explicit(c, rho, u, c->rho_bar, Erho, Em, Ee, c->stream);
}

int dgx_apply_mass(dgx_ctx *c, const double *rho, const double *in, double *out) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_mesh) return set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (!rho || !in || !out || in == out) return set_error(c, DGX_ERR_ARG, "null or aliased array");
  return mass_forward_rule(c, rho, in, out, c->stream);
}

int dgx_kinetic_mass(dgx_ctx *c, const double *rho, const double *u, double *out) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_mesh) return set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (!rho || !u || !out) return set_error(c, DGX_ERR_ARG, "null array");
  return launch_cmass(c, 1, 1.0, rho, u, out, c->stream);
}

int dgx_imex_step(dgx_ctx *c, double *rho, double *u, double *p, int nsteps, const dgx_solve_opts *opts,
                  dgx_step_info *info) {
  if (int e = ready(c)) return e;
  if (!c->has_imex) return set_error(c, DGX_ERR_STATE, "no tableau (call dgx_set_imex)");
  if (!rho || !u || !p || nsteps < 0) return set_error(c, DGX_ERR_ARG, "null state array or negative step count");
  const auto t0 = std::chrono::steady_clock::now();
  dgx_solve_opts o;
  if (opts) o = *opts;
  else dgx_default_solve_opts(&o);
  o.use_x0 = 1;
  dgx_step_info inf;
  std::memset(&inf, 0, sizeof(inf));
  ImexWS w;
  if (int e = imex_workspace(c, w)) return e;
  const long long N = c->N;
  const size_t b1 = N * sizeof(double), b3 = 3 * b1;
  const int s = c->imex_s, K = c->imex_K;
  const double dt = c->imex_dt, gm = c->bg.gamma, g = c->bg.g;
  cudaStream_t st = c->stream;
  auto cp = [&](double *d, const double *src, size_t bytes) {
    return check_cuda(c, cudaMemcpyAsync(d, src, bytes, cudaMemcpyDeviceToDevice, st), "memcpy");
  };
  int e = 0;
  count_launch(2);
  k_fill<<<grid(N), 256, 0, st>>>(N, 0.0, w.zeros);
  k_fill<<<grid(N), 256, 0, st>>>(N, 1.0, w.ones);
  if (c->nc) {  // dead cells of a non-conforming mesh carry the background at rest (no perturbation, no wind)
    if ((e = fill_dead<double>(c, rho, 1, 0.0, st, c->rho_bar)) || (e = fill_dead<double>(c, u, 3, 0.0, st)) ||
        (e = fill_dead<double>(c, p, 1, 0.0, st, c->p_bar)))
      return e;
  }
  double solve_s = 0.0;
  for (int step = 0; step < nsteps; ++step) {
    if ((e = cp(w.rn, rho, b1)) || (e = cp(w.un, u, b3)) || (e = cp(w.pn, p, b1))) return e;
    for (int l = 0; l < s; ++l) {
      double *Er = w.Ten + (size_t)9 * N * l, *Em = Er + N, *Ee = Em + 3 * N, *Im = Ee + N, *Ie = Im + 3 * N;
      if (l == 0) {
        if ((e = cp(w.rl, w.rn, b1)) || (e = cp(w.ul, w.un, b3)) || (e = cp(w.pl, w.pn, b1))) return e;
      } else {
        const double al = c->imex_At[l * s + l] * dt;
        // continuity: rho^(l) = rho^n + M^-1 dt sum a_lm Erho^(m)
        cudaMemsetAsync(w.t1, 0, b1, st);
        for (int m = 0; m < l; ++m) {
          const double *Erm = w.Ten + (size_t)9 * N * m;
          if (c->imex_A[l * s + m] != 0.0) vec_axpby<double>(N, dt * c->imex_A[l * s + m], Erm, 1.0, w.t1, st);
        }
        if ((e = mass_inverse_rule<double>(c, w.t1, w.ones, w.t2, st, 1))) return e;
        if ((e = cp(w.rl, w.rn, b1))) return e;
        vec_axpby<double>(N, 1.0, w.t2, 1.0, w.rl, st);
        // momentum right-hand side
        if ((e = mass_forward_rule(c, w.rn, w.un, w.Fs, st))) return e;
        for (int m = 0; m < l; ++m) {
          const double *Erm = w.Ten + (size_t)9 * N * m;
          if (c->imex_A[l * s + m] != 0.0) vec_axpby<double>(3 * N, dt * c->imex_A[l * s + m], Erm + N, 1.0, w.Fs, st);
          if (c->imex_At[l * s + m] != 0.0)
            vec_axpby<double>(3 * N, dt * c->imex_At[l * s + m], Erm + 5 * N, 1.0, w.Fs, st);
        }
        if ((e = cp(w.t1, w.rl, b1))) return e;
        vec_axpby<double>(N, -1.0, c->rho_bar, 1.0, w.t1, st);  // rho'^(l)
        if ((e = launch_cmass(c, 0, -g * al, w.t1, nullptr, w.t2, st))) return e;
        vec_axpby<double>(N, 1.0, w.t2, 1.0, w.Fs + 2 * N, st);
        // energy right-hand side (static part)
        if ((e = cp(w.t1, w.pn, b1))) return e;
        vec_axpby<double>(N, -1.0, c->p_bar, 1.0, w.t1, st);  // p'^n
        if ((e = launch_cmass(c, 0, 1.0 / (gm - 1.0), w.t1, nullptr, w.Gs, st))) return e;
        if ((e = launch_cmass(c, 1, 1.0, w.rn, w.un, w.t2, st))) return e;
        vec_axpby<double>(N, 1.0, w.t2, 1.0, w.Gs, st);
        for (int m = 0; m < l; ++m) {
          const double *Erm = w.Ten + (size_t)9 * N * m;
          if (c->imex_A[l * s + m] != 0.0) vec_axpby<double>(N, dt * c->imex_A[l * s + m], Erm + 4 * N, 1.0, w.Gs, st);
          if (c->imex_At[l * s + m] != 0.0)
            vec_axpby<double>(N, dt * c->imex_At[l * s + m], Erm + 8 * N, 1.0, w.Gs, st);
        }
        // W = A(rho^(l))^-1 F: the same for every fixed-point iteration of the stage
        if ((e = mass_inverse_rule<double>(c, w.Fs, w.rl, w.W, st, 3))) return e;
        // fixed-point iterations from the previous stage (ul, pl)
        for (int k = 0; k < K; ++k) {
          if ((e = dgx_set_coefficients(c, w.rl, w.pl, al, gm))) return e;
          if ((e = launch_cmass(c, 1, 1.0, w.rl, w.ul, w.t2, st))) return e;
          if ((e = cp(w.rhs, w.Gs, b1))) return e;
          vec_axpby<double>(N, -1.0, w.t2, 1.0, w.rhs, st);
          if ((e = launch_div<double>(c, w.W, w.zeros, c->pk64, w.t2, st))) return e;  // -C A^-1 F
          vec_axpby<double>(N, 1.0, w.t2, 1.0, w.rhs, st);
          if ((e = cp(w.x, w.pl, b1))) return e;
          vec_axpby<double>(N, -1.0, c->p_bar, 1.0, w.x, st);  // initial guess p'^(l,k)
          dgx_solve_info si;
          const auto ts = std::chrono::steady_clock::now();
          const int rc = solve_pressure_vx(c, w.rhs, w.x, &o, &si, w.t1);  // t1 = A^-1 B of the solution
          solve_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - ts).count();
          if (rc < 0) return rc;
          if (rc == DGX_NOT_CONVERGED) inf.status = DGX_NOT_CONVERGED;
          if (c->rec_store && c->rec_count < c->rec_cap && (++c->rec_seen % c->rec_stride) == 0) {
            double *r = c->rec_store + (size_t)c->rec_count * (4 * N + 2);
            const double sc[2] = {al, gm};
            cudaMemcpyAsync(r, c->rho64, b1, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(r + N, c->pk64, b1, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(r + 2 * N, w.rhs, b1, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(r + 3 * N, w.x, b1, cudaMemcpyDeviceToDevice, st);
            if ((e = check_cuda(c, cudaMemcpyAsync(r + 4 * N, sc, sizeof(sc), cudaMemcpyHostToDevice, st), "record")))
              return e;
            if ((e = check_cuda(c, cudaStreamSynchronize(st), "record"))) return e;
            ++c->rec_count;
          }
          inf.solves += 1;
          inf.krylov_iterations += si.iterations;
          inf.inner_iterations += si.inner_iterations;
          inf.operator_f64 += si.operator_f64;
          inf.operator_f32 += si.operator_f32;
          inf.max_relres = std::fmax(inf.max_relres, si.relres);
          if ((e = cp(w.ul, w.W, b3))) return e;
          vec_axpby<double>(3 * N, -1.0, w.t1, 1.0, w.ul, st);
          if ((e = cp(w.pl, c->p_bar, b1))) return e;
          vec_axpby<double>(N, 1.0, w.x, 1.0, w.pl, st);
        }
      }
      if (l < s - 1) {
        if ((e = launch_explicit(c, w.rl, w.ul, c->rho_bar, Er, Em, Ee, st))) return e;
        if ((e = cp(w.t2, w.pl, b1))) return e;
        vec_axpby<double>(N, -1.0, c->p_bar, 1.0, w.t2, st);
        if ((e = launch_grad<double>(c, w.t2, c->rho64, Im, st, false, 1.0))) return e;  // B_1 p'
        vec_axpby<double>(3 * N, 0.0, Im, -1.0, Im, st);                                   // -B_1 p'
        if ((e = cp(w.t1, w.rl, b1))) return e;
        vec_axpby<double>(N, -1.0, c->rho_bar, 1.0, w.t1, st);
        if ((e = launch_cmass(c, 0, -g, w.t1, nullptr, w.t2, st))) return e;              // int rho' g.phi (z)
        vec_axpby<double>(N, 1.0, w.t2, 1.0, Im + 2 * N, st);
        if ((e = launch_div<double>(c, w.ul, w.zeros, w.pl, Ie, st, 1.0))) return e;       // -C_1 u
      }
    }
    if ((e = cp(rho, w.rl, b1)) || (e = cp(u, w.ul, b3)) || (e = cp(p, w.pl, b1))) return e;
    inf.steps += 1;
  }
  if ((e = check_cuda(c, cudaStreamSynchronize(st), "IMEX step"))) return e;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  inf.seconds_solve = solve_s;
  if (info) *info = inf;
  return inf.status;
}

int dgx_imex_record(dgx_ctx *c, double *store, int capacity, int stride) {
  if (!c) return DGX_ERR_ARG;
  if (capacity < 0 || stride < 1) return set_error(c, DGX_ERR_ARG, "need capacity >= 0 and stride >= 1");
  c->rec_store = capacity > 0 ? store : nullptr;
  c->rec_cap = c->rec_store ? capacity : 0;
  c->rec_stride = stride;
  c->rec_count = 0;
  c->rec_seen = 0;
  return DGX_OK;
}

int dgx_imex_recorded(const dgx_ctx *c) { return c ? c->rec_count : -1; }

}  // extern "C"
