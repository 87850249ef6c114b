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
  return MDGP_OK;
}

int mdgp_hybrid_create(mdgp_ctx* ctx, const mdgp_macro_params* p, const double* density0, mdgp_hybrid** out) {
  if (!ctx || !p || !out || p->n_sections < 3 || !(p->dx > 0) || !(p->h0 > 0) || !(p->dt > 0) ||
      !(p->period > 0) || !(p->sf2 > 0) || !(p->l2 > 0) || !(p->sn2 >= 0) || p->inputs < 0 || p->inputs > 1)
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
    H->h[j] = p->h0 * (1.0 - 0.5 * std::cos(2.0 * M_PI * (j * p->dx) / L));
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
  for (int j = 0; j < N; ++j)
    H->G[j] = (pr[(j + 1) % N] - pr[(j + N - 1) % N]) / (2.0 * P.dx) - dP / (N * P.dx);
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
  // one batch of MD elements for the gated sections
  const int nmd = (int)md_idx.size();
  std::vector<mdgp_result> res((size_t)nmd);
  if (nmd) {
    std::vector<mdgp_element> els((size_t)nmd);
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
    }
    const double t1 = now_s();
    int st = mdgp_micro_batch(H->ctx, els.data(), nmd, res.data());
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

int mdgp_hybrid_free(mdgp_hybrid* H) {
  if (!H) return MDGP_E_ARG;
  if (H->pgp) mdgp_gp_free(H->pgp);
  delete H;
  return MDGP_OK;
}

}  // extern "C"
