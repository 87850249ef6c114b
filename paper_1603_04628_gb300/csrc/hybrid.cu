// Macro time step of the hybrid scheme (paper Algorithm 1, Sec. 2.4) on top
// of the library's GP and micro-batch entry points.
//
// One step: pressure from the equation of state (linear, or the p-GP of Sec.
// 2.4 over (h, n) fitted to pressure pre-simulations), central-difference
// gradients, the GP gate over all sections, one batched MD launch for the
// gated sections, the means of the other sections, and the continuity update
// (Eq. continuityEq).  The q-GP inputs are (h, G) or the paper's (h, n, F)
// with F = -G / n the force per unit mass on the fluid (Eq. momentumEq).  The gate depends on the database inputs only (the
// posterior variance of Eq. predVarEq does not involve the outputs, and the
// scales of Eq. d2Eq come from the inputs), so the set of sections Algorithm 1
// sends to MD is decided before any MD runs; each non-MD section's mean then
// uses the database as Algorithm 1 holds it when it reaches that section.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "mdgp.h"
#include "md_ctx.h"

struct mdgp_hybrid {
  mdgp_ctx* ctx = nullptr;
  mdgp_macro_params p;
  int N = 0;
  long long step = 0;
  long long md_total = 0;
  std::vector<double> h, n, q, sd, G;
  std::vector<int32_t> from_md;
  int D = 2;                      // q-GP input dimension: (h, G) or (h, n, F)
  std::vector<double> X, y, se;   // database: inputs row-major (D per entry), outputs, standard errors
  std::vector<double> mX;         // prior mean at the database inputs (learned mean), if any
  mdgp_mean_fn mean_fn = nullptr;
  void* mean_user = nullptr;
  mdgp_gp* pgp = nullptr;         // pressure GP over (h, n), if set
  // final snapshot of each database entry's MD run (warm_start): rows of
  // (x y z vx vy vz) as floats, fluid first, and the geometry it was taken in
  struct Snap {
    std::vector<float> xv;
    int64_t nf = 0, nw = 0;
    double h = 0.0;
    double g = 0.0;   // the run's force per unit mass on the fluid
  };
  std::vector<Snap> snaps;
};

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

double sn2_for_step(const mdgp_hybrid* H) {
  if (H->p.sn2_from_data && !H->se.empty()) {
    double m = 0.0;
    for (double v : H->se) m += v;
    m /= (double)H->se.size();
    return m * m;
  }
  return H->p.sn2;
}

// Prior mean at rows of Xq (zero without a mean function).
int prior_mean(mdgp_hybrid* H, const double* Xq, int64_t m, std::vector<double>& out) {
  out.assign((size_t)m, 0.0);
  if (!H->mean_fn || m == 0) return MDGP_OK;
  return H->mean_fn(H->mean_user, Xq, m, out.data());
}

// Natural scale of each q-GP input, used where the database has no spread in
// it (all h equal; the uniform gradient of the first steps; uniform density):
// h0 / 2 for h, the forcing gradient amplitude dP_amp / L for G (and that
// over n0 for F), a tenth of n0 for n.
void fallback_scales(const mdgp_hybrid* H, double* fb) {
  const double L = H->p.n_sections * H->p.dx;
  const double g = H->p.dP_amp > 0 ? H->p.dP_amp / L : 1.0;
  fb[0] = 0.5 * H->p.h0;
  if (H->D == 2) {
    fb[1] = g;
  } else {
    fb[1] = 0.1 * H->p.eos_n0;
    fb[2] = g / H->p.eos_n0;
  }
}

// Section j's q-GP input row.
void input_row(const mdgp_hybrid* H, int j, double* x) {
  x[0] = H->h[j];
  if (H->D == 2) {
    x[1] = H->G[j];
  } else {
    x[1] = H->n[j];
    x[2] = -H->G[j] / H->n[j];
  }
}

// q-GP hyperparameters of a step (Sec. 2.3 values; sn2 as the step fixes it)
// with the per-dimension fallback scales; fb holds the fallbacks.
mdgp_gp_params step_params(const mdgp_hybrid* H, double sn2, double* fb) {
  mdgp_gp_params gp;
  std::memset(&gp, 0, sizeof(gp));
  gp.sf2 = H->p.sf2;
  gp.l2 = H->p.l2;
  gp.sn2 = sn2;
  fallback_scales(H, fb);
  gp.fallback_scale = 1.0;
  gp.fallback_scales = fb;
  return gp;
}

// Factor for the database inputs X rows [0, M) (no outputs: the gate needs
// none) and the posterior variances at the rows of Xq.
int gate_fit(mdgp_hybrid* H, const std::vector<double>& X, int64_t M, double sn2, const double* Xq, int64_t m,
             double* var, mdgp_gp** out) {
  double fb[3];
  const mdgp_gp_params gp = step_params(H, sn2, fb);
  mdgp_gp* g = nullptr;
  int st = mdgp_gp_fit_inputs(H->ctx, M ? X.data() : nullptr, M, H->D, &gp, &g);
  if (st) return st;
  st = mdgp_gp_predict(g, Xq, m, nullptr, nullptr, var);
  if (st) { mdgp_gp_free(g); return st; }
  *out = g;
  return MDGP_OK;
}

// Means at the rows of Xq from a gate factor whose inputs are the database's
// first M rows: the outputs y (and prior means mX) of those rows are added
// on the same factor, so the result is that of a fresh fit to (X, y).
int factor_means(mdgp_hybrid* H, mdgp_gp* g, const std::vector<double>& y, const std::vector<double>& mX,
                 int64_t M, const double* Xq, int64_t m, double* mean) {
  int st = mdgp_gp_set_outputs(g, M ? y.data() : nullptr, (H->mean_fn && M) ? mX.data() : nullptr);
  if (st) return st;
  std::vector<double> mq;
  if ((st = prior_mean(H, Xq, m, mq))) return st;
  return mdgp_gp_predict(g, Xq, m, H->mean_fn ? mq.data() : nullptr, mean, nullptr);
}

// Eq. d2Eq scales of the database inputs X (M rows of D): the mean of
// |x_ik - x_jk| over all pairs i < j, the fallback where it is undefined.
void host_scales(const mdgp_hybrid* H, const std::vector<double>& X, int64_t M, double* sc) {
  double fb[3];
  fallback_scales(H, fb);
  const int D = H->D;
  for (int d = 0; d < D; ++d) {
    double tot = 0.0;
    for (int64_t i = 0; i < M; ++i)
      for (int64_t j = i + 1; j < M; ++j) tot += std::fabs(X[(size_t)D * i + d] - X[(size_t)D * j + d]);
    const double mean = M > 1 ? tot / (0.5 * (double)M * (double)(M - 1)) : 0.0;
    sc[d] = mean > 0.0 ? mean : fb[d];
  }
}

// The entry x_in among the first M database entries with a snapshot taken
// at channel height h that maximises K(x_in, x*) for the squared-
// exponential kernel, i.e. the smallest scaled distance (Eq. d2Eq) to x*;
// -1 when there is none (the run then starts from the lattice).
int64_t most_correlated(const mdgp_hybrid* H, int64_t M, const double* sc, const double* xs, double h) {
  int64_t best = -1;
  double bd = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    const mdgp_hybrid::Snap& S = H->snaps[(size_t)i];
    if (S.xv.empty() || std::fabs(S.h - h) > 1e-9) continue;
    double d2 = 0.0;
    for (int d = 0; d < H->D; ++d) {
      const double t = (H->X[(size_t)H->D * i + d] - xs[d]) / sc[d];
      d2 += t * t;
    }
    if (best < 0 || d2 < bd) { best = i; bd = d2; }
  }
  return best;
}

// One group of MD runs sharing a step count, through the plan / launch /
// results / state entry points (with mdgp_micro_batch's rerun on list
// overflow); when keep is set, each run's final state becomes a snapshot.
int run_group(mdgp_hybrid* H, const std::vector<mdgp_element>& els, const std::vector<mdgp_start>& starts,
              mdgp_result* res, bool keep, std::vector<mdgp_hybrid::Snap>* out) {
  mdgp_ctx* ctx = H->ctx;
  const int64_t n = (int64_t)els.size();
  const int32_t cap0 = ctx->params.list_capacity;
  int st = MDGP_OK;
  for (int attempt = 0; attempt < 3; ++attempt) {
    int64_t atoms = 0;
    st = mdgp_micro_plan_from(ctx, els.data(), n, starts.data(), &atoms);
    if (!st) st = mdgp_micro_launch(ctx);
    if (!st) st = mdgp_micro_results(ctx, res, n);
    if (st) break;
    bool overflow = false;
    for (int64_t k = 0; k < n; ++k) overflow |= res[k].status == MDGP_E_OVERFLOW;
    if (!overflow || attempt == 2) {
      if (keep) {
        std::vector<double> x((size_t)3 * atoms), v((size_t)3 * atoms);
        st = mdgp_micro_state(ctx, x.data(), v.data(), atoms);
        if (st) break;
        out->resize((size_t)n);
        int64_t off = 0;
        for (int64_t k = 0; k < n; ++k) {
          mdgp_hybrid::Snap& S = (*out)[(size_t)k];
          S.nf = res[k].n_fluid;
          S.nw = res[k].n_wall;
          S.h = els[(size_t)k].h;
          S.g = els[(size_t)k].density > 0.0 ? els[(size_t)k].g_ext - els[(size_t)k].dpdx / els[(size_t)k].density
                                               : els[(size_t)k].g_ext;
          const int64_t m = S.nf + S.nw;
          S.xv.resize((size_t)6 * m);
          for (int64_t a = 0; a < m; ++a)
            for (int d = 0; d < 3; ++d) {
              S.xv[(size_t)6 * a + d] = (float)x[(size_t)3 * (off + a) + d];
              S.xv[(size_t)6 * a + 3 + d] = (float)v[(size_t)3 * (off + a) + d];
            }
          off += m;
        }
      }
      break;
    }
    ctx->params.list_capacity = 2 * (ctx->params.list_capacity > 0 ? ctx->params.list_capacity : 128);
    ctx->planned = false;
  }
  ctx->params.list_capacity = cap0;
  ctx->planned = false;
  return st;
}

// The gate factors of one step; freed when the step ends.
struct Factors {
  std::vector<mdgp_gp*> g;
  ~Factors() {
    for (mdgp_gp* x : g)
      if (x) mdgp_gp_free(x);   // null: not kept (memory budget)
  }
};

}  // namespace

extern "C" {

// Algorithm 1's pseudoMD: the 1D channel-flow start-up with Navier slip
// (Sec. 2.4), nodes y_i = i h / n, i = 0..n.
namespace {

// Solve the tridiagonal system a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i
// (Thomas algorithm; a_0 and c_{n-1} unused); d is overwritten by x.
void thomas(const std::vector<double>& a, const std::vector<double>& b, const std::vector<double>& c,
            std::vector<double>& d, std::vector<double>& w) {
  const size_t n = b.size();
  w.assign(n, 0.0);
  double beta = b[0];
  d[0] /= beta;
  for (size_t i = 1; i < n; ++i) {
    w[i] = c[i - 1] / beta;
    beta = b[i] - a[i] * w[i];
    d[i] = (d[i] - a[i] * d[i - 1]) / beta;
  }
  for (size_t i = n - 1; i-- > 0;) d[i] -= w[i + 1] * d[i + 1];
}

}  // namespace

int mdgp_pseudo_md(double h, double nu, double slip, double g_from, double g_to, int32_t from_rest,
                   double q_scale, double eps_q, double* t_s) {
  if (!t_s || !(h > 0) || !(nu > 0) || !(q_scale > 0) || !(eps_q > 0) || !(h + 2.0 * slip > 0)) return MDGP_E_ARG;
  if (slip < 0.0) {   // no-slip planes -slip inside each wall: the flowing width h + 2 slip
    h += 2.0 * slip;
    slip = 0.0;
  }
  constexpr int n = 64;
  const double dy = h / n;
  const double k = nu / (dy * dy);
  // rows of the operator nu d2/dy2 on u_0..u_n: interior (1, -2, 1) k; a
  // wall node with slip takes its ghost u_-1 = u_1 - 2 dy u_0 / slip,
  // giving (2 u_1 - (2 + 2 dy / slip) u_0) k; without slip u_0 = 0
  std::vector<double> lo(n + 1, k), di(n + 1, -2.0 * k), up(n + 1, k);
  const bool dirichlet = slip == 0.0;
  if (!dirichlet) {
    di[0] = di[n] = -(2.0 + 2.0 * dy / slip) * k;
    up[0] = 2.0 * k;
    lo[n] = 2.0 * k;
  }
  auto flow = [&](const std::vector<double>& u) {
    double s = 0.5 * (u[0] + u[n]);
    for (int i = 1; i < n; ++i) s += u[i];
    return q_scale * s * dy;
  };
  // steady states: nu u'' = -g
  std::vector<double> w;
  auto steady = [&](double g, std::vector<double>& u) {
    std::vector<double> a(lo), b(di), c(up);
    u.assign(n + 1, -g);
    if (dirichlet) {
      b[0] = b[n] = 1.0; c[0] = a[n] = 0.0; u[0] = u[n] = 0.0;
    }
    thomas(a, b, c, u, w);
  };
  std::vector<double> u, uinf;
  steady(g_to, uinf);
  if (from_rest) u.assign(n + 1, 0.0);
  else steady(g_from, u);
  const double qinf = flow(uinf);
  const double tau = h * h / (nu * M_PI * M_PI);
  const double dt = tau / 1000.0;
  // implicit Euler: (I - dt A) u' = u + dt g
  std::vector<double> a(n + 1), b(n + 1), c(n + 1), r(n + 1);
  for (int i = 0; i <= n; ++i) { a[i] = -dt * lo[i]; b[i] = 1.0 - dt * di[i]; c[i] = -dt * up[i]; }
  if (dirichlet) { b[0] = b[n] = 1.0; c[0] = a[n] = 0.0; }
  double t = 0.0;
  for (long it = 0; it <= 1000000; ++it) {
    if (std::fabs(flow(u) - qinf) <= eps_q) {
      *t_s = t;
      return MDGP_OK;
    }
    if (it == 1000000) break;
    for (int i = 0; i <= n; ++i) r[i] = u[i] + dt * g_to;
    if (dirichlet) r[0] = r[n] = 0.0;
    thomas(a, b, c, r, w);
    u.swap(r);
    t += dt;
  }
  return MDGP_E_LIMIT;
}

int mdgp_macro_params_default(mdgp_macro_params* p) {
  if (!p) return MDGP_E_ARG;
  std::memset(p, 0, sizeof(*p));
  p->n_sections = 200;
  p->dx = 50.0;
  p->h0 = 12.0;
  p->Lx = 10.0;
  p->Lz = 10.0;
  p->eos_K = 10.0;
  p->eos_n0 = 0.8;
  p->dP_amp = 400.0;
  p->period = 1000.0;
  p->dt = 20.0;
  p->T = 1.1;
  p->md_steps_eq = 2000;
  p->md_steps_sample = 3000;
  p->seed = 20160315ULL;
  p->sf2 = 100.0;
  p->l2 = 1.0;
  p->sn2 = 0.25;
  p->sn2_from_data = 0;
  p->inputs = 0;
  p->warm_start = 0;
  p->md_steps_eq_warm = 0;
  p->h_amp = 0.5;
  return MDGP_OK;
}

int mdgp_hybrid_create(mdgp_ctx* ctx, const mdgp_macro_params* p, const double* density0, mdgp_hybrid** out) {
  if (!ctx || !p || !out || p->n_sections < 3 || !(p->dx > 0) || !(p->h0 > 0) || !(p->dt > 0) ||
      !(p->period > 0) || !(p->sf2 > 0) || !(p->l2 > 0) || !(p->sn2 >= 0) || p->inputs < 0 || p->inputs > 1 ||
      !(p->h_amp >= 0.0 && p->h_amp < 1.0))
    return MDGP_E_ARG;
  *out = nullptr;
  mdgp_hybrid* H = new (std::nothrow) mdgp_hybrid();
  if (!H) return MDGP_E_NOMEM;
  H->ctx = ctx;
  H->p = *p;
  H->N = p->n_sections;
  H->D = p->inputs == 1 ? 3 : 2;
  const double L = H->N * p->dx;
  H->h.resize(H->N);
  H->n.resize(H->N);
  for (int j = 0; j < H->N; ++j) {
    H->h[j] = p->h0 * (1.0 - p->h_amp * std::cos(2.0 * M_PI * (j * p->dx) / L));
    H->n[j] = density0 ? density0[j] : p->eos_n0;
  }
  H->q.assign(H->N, 0.0);
  H->sd.assign(H->N, 0.0);
  H->G.assign(H->N, 0.0);
  H->from_md.assign(H->N, 0);
  *out = H;
  return MDGP_OK;
}

int mdgp_hybrid_set_mean(mdgp_hybrid* H, mdgp_mean_fn fn, void* user) {
  if (!H) return MDGP_E_ARG;
  H->mean_fn = fn;
  H->mean_user = user;
  // prior mean at the existing database inputs
  const int64_t M = (int64_t)H->y.size();
  return prior_mean(H, H->X.data(), M, H->mX);
}

static int mlp_mean_fn(void* user, const double* x, int64_t m, double* out) {
  return mdgp_mlp_predict((mdgp_mlp*)user, x, m, out);
}

int mdgp_hybrid_set_mlp_mean(mdgp_hybrid* H, mdgp_mlp* m) {
  if (!H || (m && H->D != 2)) return MDGP_E_ARG;   // the network takes 2 inputs
  return m ? mdgp_hybrid_set_mean(H, mlp_mean_fn, m) : mdgp_hybrid_set_mean(H, nullptr, nullptr);
}

int mdgp_hybrid_step(mdgp_hybrid* H, double sigma_t, mdgp_hybrid_stats* stats) {
  if (!H || !(sigma_t >= 0)) return MDGP_E_ARG;
  const int N = H->N;
  const mdgp_macro_params& P = H->p;
  double t_gp = 0.0, t_md = 0.0, t0 = now_s();
  H->step += 1;
  const double t = H->step * P.dt;
  // pressure (equation of state or p-GP mean), its gradient (central
  // differences, periodic) and the forcing
  const double dP = P.dP_amp * std::sin(2.0 * M_PI * t / P.period);
  std::vector<double> pr((size_t)N);
  if (H->pgp) {
    std::vector<double> Xp((size_t)2 * N), pv((size_t)N);
    for (int j = 0; j < N; ++j) { Xp[2 * j] = H->h[j]; Xp[2 * j + 1] = H->n[j]; }
    int st = mdgp_gp_predict(H->pgp, Xp.data(), N, nullptr, pr.data(), pv.data());
    if (st) return st;
  } else {
    for (int j = 0; j < N; ++j) pr[j] = P.eos_K * (H->n[j] - P.eos_n0);
  }
  // Eq. momentumEq: every fluid atom feels F_j = F_ext - (m / rho_j) p'_j with
  // the external force F_ext uniform over the channel; the inlet-outlet
  // difference dP(t) sets it at the initial density, F_ext = dP / (L n0).
  // G_j = p'_j - n_j F_ext is the gradient an element is given (F = -G / n).
  const double f_ext = dP / (N * P.dx * P.eos_n0);
  for (int j = 0; j < N; ++j)
    H->G[j] = (pr[(j + 1) % N] - pr[(j + N - 1) % N]) / (2.0 * P.dx) - H->n[j] * f_ext;
  const double sn2 = sn2_for_step(H);
  const int D = H->D;
  std::vector<double> Xq((size_t)D * N);
  for (int j = 0; j < N; ++j) input_row(H, j, Xq.data() + (size_t)D * j);
  // gate pass: variance on the inputs only, appending gated inputs in order.
  // sigma_t <= 0 sends every section to MD whatever the variance (the
  // reference run), so no GP work is done then.
  const int64_t M0 = (int64_t)H->y.size();
  std::vector<double> Xv(H->X), mv(H->mX);
  std::vector<int> md_idx;
  std::vector<double> mean((size_t)N), var((size_t)N);
  int j0 = 0;
  if (!(sigma_t > 0.0)) {
    for (int j = 0; j < N; ++j) {
      md_idx.push_back(j);
      H->sd[j] = NAN;
      if (H->mean_fn) {
        std::vector<double> mq;
        int st2 = prior_mean(H, Xq.data() + (size_t)D * j, 1, mq);
        if (st2) return st2;
        mv.push_back(mq[0]);
      }
    }
    j0 = N;
  }
  // factors.g[k]: the factor of the database with the first k gated inputs
  // appended, the one every later mean up to the next MD section uses; null
  // where keeping it would pass the memory budget
  Factors factors;
  const long long cache_mb = P.factor_cache_mb ? P.factor_cache_mb : 4096;
  const long long keep_bytes = P.factor_cache_mb < 0 ? -1 : cache_mb << 20;
  long long kept = 0;
  while (j0 < N) {
    const int64_t Mv = (int64_t)(Xv.size() / D);
    mdgp_gp* g = nullptr;
    int st = gate_fit(H, Xv, Mv, sn2, Xq.data() + (size_t)D * j0, N - j0, var.data() + j0, &g);
    if (st) return st;
    const long long Mp = (Mv + 31) / 32 * 32, bytes = Mp * Mp * (long long)sizeof(double);
    if (kept + bytes <= keep_bytes) {
      kept += bytes;
      factors.g.push_back(g);
    } else {
      mdgp_gp_free(g);
      factors.g.push_back(nullptr);
    }
    int j = j0;
    for (; j < N; ++j) {
      H->sd[j] = std::sqrt(var[j]);
      if (H->sd[j] > sigma_t) break;
    }
    if (j == N) break;
    md_idx.push_back(j);
    for (int d = 0; d < D; ++d) Xv.push_back(Xq[(size_t)D * j + d]);
    if (H->mean_fn) {
      std::vector<double> mq;
      int st2 = prior_mean(H, Xq.data() + (size_t)D * j, 1, mq);
      if (st2) return st2;
      mv.push_back(mq[0]);
    }
    j0 = j + 1;
  }
  t_gp += now_s() - t0;
  // one batch of MD elements for the gated sections (two with warm starts:
  // the runs from snapshots equilibrate for fewer steps)
  const int nmd = (int)md_idx.size();
  std::vector<mdgp_result> res((size_t)nmd);
  std::vector<mdgp_hybrid::Snap> new_snaps;
  int n_warm = 0;
  long long eq_used = 0;
  if (nmd) {
    std::vector<mdgp_element> els((size_t)nmd);
    std::vector<mdgp_start> starts((size_t)nmd);
    std::vector<double> sc((size_t)D, 1.0);
    if (P.warm_start && M0 > 0) host_scales(H, H->X, M0, sc.data());
    const long long eq_warm = P.md_steps_eq_warm > 0 ? P.md_steps_eq_warm : P.md_steps_eq / 4;
    // with pseudoMD the warm group equilibrates for the longest start-up
    // time t_s of its runs (one plan shares its step count), in MD steps,
    // within [eq_warm, md_steps_eq]
    const double sn2 = sn2_for_step(H);
    const double eps_q = P.pseudo_eps_q > 0.0 ? P.pseudo_eps_q : 0.25 * std::sqrt(sn2);
    long long eq_pseudo = eq_warm;
    for (int k = 0; k < nmd; ++k) {
      const int j = md_idx[k];
      mdgp_element& e = els[k];
      std::memset(&e, 0, sizeof(e));
      e.h = H->h[j];
      e.dpdx = H->G[j];
      e.density = H->n[j];
      e.T = P.T;
      e.steps_eq = P.md_steps_eq;
      e.steps_sample = P.md_steps_sample;
      e.Lx = P.Lx;
      e.Lz = P.Lz;
      e.g_ext = 0.0;
      e.seed = P.seed;
      e.id = (int32_t)(H->md_total + k);
      std::memset(&starts[k], 0, sizeof(mdgp_start));
      if (P.warm_start && M0 > 0) {
        const int64_t in = most_correlated(H, M0, sc.data(), Xq.data() + (size_t)D * j, H->h[j]);
        if (in >= 0) {
          const mdgp_hybrid::Snap& S = H->snaps[(size_t)in];
          starts[k].xv = S.xv.data();
          starts[k].n_fluid = S.nf;
          starts[k].n_wall = S.nw;
          starts[k].h = S.h;
          starts[k].Lx = P.Lx;
          starts[k].Lz = P.Lz;
          e.steps_eq = eq_warm;
          if (P.pseudo_nu > 0.0 && eps_q > 0.0) {
            const double g = e.density > 0.0 ? -e.dpdx / e.density : 0.0;
            double ts = 0.0;
            const int ps = mdgp_pseudo_md(e.h, P.pseudo_nu, P.pseudo_slip, S.g, g, 0,
                                          H->ctx->params.mass * e.density * P.Lz, eps_q, &ts);
            const long long want = ps == MDGP_OK ? (long long)std::ceil(ts / H->ctx->params.dt) : P.md_steps_eq;
            eq_pseudo = std::max(eq_pseudo, std::min<long long>(std::max<long long>(want, eq_warm), P.md_steps_eq));
          }
        }
      }
    }
    const double t1 = now_s();
    int st = MDGP_OK;
    if (!P.warm_start) {
      st = mdgp_micro_batch(H->ctx, els.data(), nmd, res.data());
    } else {
      // the warm group, then the cold group (a warm start the library
      // declines runs from the lattice with the warm group's equilibration)
      new_snaps.resize((size_t)nmd);
      for (int warm = 1; warm >= 0 && !st; --warm) {
        std::vector<int> idx;
        for (int k = 0; k < nmd; ++k)
          if ((starts[k].xv != nullptr) == (warm == 1)) idx.push_back(k);
        if (idx.empty()) continue;
        std::vector<mdgp_element> ge;
        std::vector<mdgp_start> gs;
        for (int k : idx) {
          ge.push_back(els[k]);
          if (warm) ge.back().steps_eq = eq_pseudo;
          gs.push_back(starts[k]);
        }
        if (warm) eq_used = eq_pseudo;
        std::vector<mdgp_result> gr(idx.size());
        std::vector<mdgp_hybrid::Snap> snaps;
        st = run_group(H, ge, gs, gr.data(), true, &snaps);
        for (size_t q = 0; q < idx.size() && !st; ++q) {
          res[(size_t)idx[q]] = gr[q];
          new_snaps[(size_t)idx[q]] = std::move(snaps[q]);
          n_warm += gr[q].start > 0 ? 1 : 0;
        }
      }
    }
    t_md += now_s() - t1;
    if (st) return st;
  }
  H->md_total += nmd;
  // means: each run of non-MD sections uses the database with every earlier
  // MD result of this step appended, i.e. the inputs of gate factor k (k
  // results appended) with their outputs added
  const double t2 = now_s();
  int k = 0, j = 0;
  while (j < N) {
    if (k < nmd && md_idx[k] == j) {
      H->q[j] = res[k].q;
      H->from_md[j] = 1;
      for (int d = 0; d < D; ++d) H->X.push_back(Xq[(size_t)D * j + d]);
      H->y.push_back(res[k].q);
      H->se.push_back(res[k].q_se);
      H->snaps.emplace_back();
      if (P.warm_start) H->snaps.back() = std::move(new_snaps[(size_t)k]);
      if (H->mean_fn) H->mX.push_back(mv[(size_t)M0 + k]);
      ++k;
      ++j;
      continue;
    }
    const int jend = (k < nmd) ? md_idx[k] : N;
    const int64_t M = (int64_t)H->y.size();
    if (k >= (int)factors.g.size()) return MDGP_E_STATE;   // the gate scanned every section it factored for
    mdgp_gp* g = factors.g[k];
    mdgp_gp* own = nullptr;
    if (!g) {
      // not kept: the same inputs factored again (the scales and the factor
      // are deterministic, so it is the gate's factor bit for bit)
      double fb[3];
      const mdgp_gp_params gp = step_params(H, sn2, fb);
      int st0 = mdgp_gp_fit_inputs(H->ctx, M ? H->X.data() : nullptr, M, D, &gp, &own);
      if (st0) return st0;
      g = own;
    }
    int st = factor_means(H, g, H->y, H->mX, M, Xq.data() + (size_t)D * j, jend - j, mean.data() + j);
    if (own) mdgp_gp_free(own);
    if (st) return st;
    for (int i = j; i < jend; ++i) {
      H->q[i] = mean[i];
      H->from_md[i] = 0;
    }
    j = jend;
  }
  t_gp += now_s() - t2;
  // continuity (Eq. continuityEq, central differences)
  std::vector<double> nn(H->n);
  for (int i = 0; i < N; ++i) {
    const double A = H->h[i] * P.Lz;
    nn[i] = H->n[i] - P.dt / A * (H->q[(i + 1) % N] - H->q[(i + N - 1) % N]) / (2.0 * P.dx);
  }
  H->n.swap(nn);
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->step = H->step;
    stats->t = t;
    stats->md_runs = nmd;
    stats->md_warm = n_warm;
    stats->md_steps_eq_warm = eq_used;
    stats->md_runs_total = H->md_total;
    stats->db_size = (int64_t)H->y.size();
    double qs = 0.0, mx = 0.0;
    for (int i = 0; i < N; ++i) { qs += H->q[i]; mx = std::fmax(mx, H->sd[i]); }
    stats->q_mean = qs / N;
    stats->max_sd = mx;
    stats->gp_seconds = t_gp;
    stats->md_seconds = t_md;
    long long atoms = 0;
    for (auto& r : res) atoms += r.n_fluid + r.n_wall;
    stats->md_atoms = atoms;
  }
  return MDGP_OK;
}

int mdgp_hybrid_state(const mdgp_hybrid* H, double* density, double* q, double* sd, int32_t* from_md,
                      double* G) {
  if (!H) return MDGP_E_ARG;
  for (int j = 0; j < H->N; ++j) {
    if (density) density[j] = H->n[j];
    if (q) q[j] = H->q[j];
    if (sd) sd[j] = H->sd[j];
    if (from_md) from_md[j] = H->from_md[j];
    if (G) G[j] = H->G[j];
  }
  return MDGP_OK;
}

int mdgp_hybrid_database(const mdgp_hybrid* H, double* X, double* y, double* se, int64_t cap, int64_t* M) {
  if (!H || !M) return MDGP_E_ARG;
  const int64_t m = (int64_t)H->y.size();
  *M = m;
  if (cap < m) return (X || y || se) ? MDGP_E_ARG : MDGP_OK;
  for (int64_t i = 0; i < m; ++i) {
    if (X) for (int d = 0; d < H->D; ++d) X[H->D * i + d] = H->X[(size_t)H->D * i + d];
    if (y) y[i] = H->y[i];
    if (se) se[i] = H->se[i];
  }
  return MDGP_OK;
}

int mdgp_hybrid_set_pressure(mdgp_hybrid* H, const double* X, const double* y, int64_t M, double sf2, double l2,
                             double sn2) {
  if (!H || M < 0 || (M > 0 && (!X || !y)) || (M > 0 && (!(sf2 > 0) || !(l2 > 0) || !(sn2 >= 0))))
    return MDGP_E_ARG;
  if (H->pgp) { mdgp_gp_free(H->pgp); H->pgp = nullptr; }
  if (M == 0) return MDGP_OK;   // back to the linear equation of state
  mdgp_gp_params gp;
  std::memset(&gp, 0, sizeof(gp));
  gp.sf2 = sf2;
  gp.l2 = l2;
  gp.sn2 = sn2;
  const double fb[2] = {0.5 * H->p.h0, 0.1 * H->p.eos_n0};
  gp.fallback_scale = 1.0;
  gp.fallback_scales = fb;
  return mdgp_gp_fit(H->ctx, X, y, M, 2, &gp, nullptr, &H->pgp);
}

int mdgp_hybrid_set_database(mdgp_hybrid* H, const double* X, const double* y, const double* se, int64_t M) {
  if (!H || M < 0 || (M > 0 && (!X || !y))) return MDGP_E_ARG;
  std::vector<double> nX(X, X + (size_t)H->D * M), ny(y, y + M), nse((size_t)M, 0.0), mX;
  if (se) nse.assign(se, se + M);
  const int st = prior_mean(H, nX.data(), M, mX);
  if (st) return st;
  H->X.swap(nX);
  H->y.swap(ny);
  H->se.swap(nse);
  H->mX.swap(mX);
  H->snaps.assign((size_t)M, mdgp_hybrid::Snap());
  return MDGP_OK;
}

// Database file (Sec. 3.3: a case starts from the database an earlier case
// ended with): little-endian host layout.
//   char magic[8] = "MDGPDB1"; int32 D; int32 with_snapshots; int64 M;
//   double X[M * D], y[M], se[M];
//   then with_snapshots: per entry int64 n_fluid, n_wall; double h, g;
//   float xv[6 * (n_fluid + n_wall)] (n_fluid = n_wall = 0: no snapshot).
static const char kDbMagic[8] = {'M', 'D', 'G', 'P', 'D', 'B', '1', '\0'};

int mdgp_hybrid_save(const mdgp_hybrid* H, const char* path, int32_t with_snapshots) {
  if (!H || !path) return MDGP_E_ARG;
  FILE* f = std::fopen(path, "wb");
  if (!f) return MDGP_E_ARG;
  const int32_t D = H->D, ws = with_snapshots ? 1 : 0;
  const int64_t M = (int64_t)H->y.size();
  bool ok = std::fwrite(kDbMagic, 1, 8, f) == 8 && std::fwrite(&D, 4, 1, f) == 1 && std::fwrite(&ws, 4, 1, f) == 1 &&
            std::fwrite(&M, 8, 1, f) == 1;
  ok = ok && (M == 0 || (std::fwrite(H->X.data(), 8, (size_t)D * M, f) == (size_t)D * M &&
                         std::fwrite(H->y.data(), 8, (size_t)M, f) == (size_t)M &&
                         std::fwrite(H->se.data(), 8, (size_t)M, f) == (size_t)M));
  for (int64_t i = 0; ok && ws && i < M; ++i) {
    const mdgp_hybrid::Snap& S = H->snaps[(size_t)i];
    const int64_t nf = S.xv.empty() ? 0 : S.nf, nw = S.xv.empty() ? 0 : S.nw;
    const size_t nv = (size_t)6 * (nf + nw);
    ok = std::fwrite(&nf, 8, 1, f) == 1 && std::fwrite(&nw, 8, 1, f) == 1 && std::fwrite(&S.h, 8, 1, f) == 1 &&
         std::fwrite(&S.g, 8, 1, f) == 1 && (nv == 0 || std::fwrite(S.xv.data(), 4, nv, f) == nv);
  }
  ok = std::fclose(f) == 0 && ok;
  return ok ? MDGP_OK : MDGP_E_ARG;
}

int mdgp_hybrid_load(mdgp_hybrid* H, const char* path) {
  if (!H || !path) return MDGP_E_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return MDGP_E_ARG;
  char magic[8];
  int32_t D = 0, ws = 0;
  int64_t M = -1;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kDbMagic, 8) == 0 &&
            std::fread(&D, 4, 1, f) == 1 && std::fread(&ws, 4, 1, f) == 1 && std::fread(&M, 8, 1, f) == 1 &&
            D == H->D && M >= 0 && M < (int64_t(1) << 31);
  std::vector<double> X, y, se;
  std::vector<mdgp_hybrid::Snap> snaps;
  if (ok) {
    X.resize((size_t)D * M);
    y.resize((size_t)M);
    se.resize((size_t)M);
    ok = M == 0 || (std::fread(X.data(), 8, X.size(), f) == X.size() && std::fread(y.data(), 8, y.size(), f) == y.size() &&
                    std::fread(se.data(), 8, se.size(), f) == se.size());
  }
  snaps.resize(ok ? (size_t)M : 0);
  for (int64_t i = 0; ok && ws && i < M; ++i) {
    mdgp_hybrid::Snap& S = snaps[(size_t)i];
    int64_t nf = 0, nw = 0;
    ok = std::fread(&nf, 8, 1, f) == 1 && std::fread(&nw, 8, 1, f) == 1 && std::fread(&S.h, 8, 1, f) == 1 &&
         std::fread(&S.g, 8, 1, f) == 1 && nf >= 0 && nw >= 0 && nf + nw < (int64_t(1) << 31);
    if (!ok) break;
    S.nf = nf;
    S.nw = nw;
    S.xv.resize((size_t)6 * (nf + nw));
    ok = S.xv.empty() || std::fread(S.xv.data(), 4, S.xv.size(), f) == S.xv.size();
  }
  std::fclose(f);
  if (!ok) return MDGP_E_ARG;
  std::vector<double> mX;
  const int st = prior_mean(H, X.data(), M, mX);
  if (st) return st;
  H->X.swap(X);
  H->y.swap(y);
  H->se.swap(se);
  H->mX.swap(mX);
  H->snaps.swap(snaps);
  return MDGP_OK;
}

int mdgp_hybrid_free(mdgp_hybrid* H) {
  if (!H) return MDGP_E_ARG;
  if (H->pgp) mdgp_gp_free(H->pgp);
  delete H;
  return MDGP_OK;
}

}  // extern "C"
