// C ABI entry points (include/stst.h) and the host-side planner of the sum-factorised mat-vec.
//
// The system matrix (Eq. syst_mat) is a short sum of Kronecker products of banded 1D matrices:
//   A = M_s (x) L_t + nu^2 B_s (x) M_t + nu L_s (x) (W_t + W_t^*),
// B_s = sum_l J_l (x) M_rest + 2 sum_{l<k} L_l (x) L_k (x) M_rest (integration by parts with the
// Dirichlet-reduced basis), L_s = sum_l L_l (x) M_rest, W_t + W_t^* = i (K_t - K_t^T).
// A separable potential V = sum_r prod_l v_{r,l} adds
//   sum_{r,r'} M_{v_r v_r'} (x) M_t + sum_r M_{v_r} (x) (W + W^*) - nu sum_{r,l} (K2S_{v_rl} at l, M_{v_r} elsewhere) (x) M_t.
// The planner turns the term list into levels of mode applications with shared intermediates:
// level 0 applies each distinct matrix of the first mode once; later levels group the terms by the
// matrices they still need. The mode order with the fewest band applications is chosen.
#include "common.cuh"
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>

namespace {

struct Term {
  double coef;
  int m[STST_MAXD + 1];  // matrix id per direction (0 = time)
};

enum { TM_L = 0, TM_M = 1, TM_KA = 2 };            // time matrix ids
enum { SM_M = 0, SM_L = 1, SM_J = 2, SM_K2S = 3 };  // spatial ids (weighted ones appended)

struct WeightReg {
  // per direction: weight id -> (device array or null for 1, M id, K2S id)
  std::vector<const double *> ptr;
  std::vector<int> mid, kid;
};

int alloc(void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_OOM;
  }
  return STST_OK;
}

int add_band(stst_problem *h, int l, int kind, const double *weight) {
  const DirInfo &D = h->dir[l];
  BandMat B;
  B.n = D.n;
  B.p = D.p;
  STST_TRY(alloc((void **)&B.d, sizeof(double) * B.n * (2 * B.p + 1)));
  float *f32 = nullptr;
  int s = launch_assemble_band(kind, D.p, D.n_el, D.len, D.nq, D.off, D.n, D.n, weight, B.d, h->stream);
  if (s == STST_OK) s = alloc((void **)&f32, sizeof(float) * B.n * (2 * B.p + 1));
  if (s == STST_OK) s = launch_to_f32(B.d, f32, (long long)B.n * (2 * B.p + 1), h->stream);
  if (s != STST_OK) {
    cudaFree(B.d);
    cudaFree(f32);
    return s;
  }
  h->mats[l].push_back(B);
  h->mats32[l].push_back(f32);
  return (int)h->mats[l].size() - 1;
}

// ---- planner ---------------------------------------------------------------------------------------
struct LevelSpec {
  int mode;
  std::vector<std::pair<int, int>> apps;  // (input index, matrix id)
  std::vector<std::vector<double>> coef;  // [app][out]
  int n_in, n_out;
};

// Build the levels for a given mode order; returns total band work (sum over contributions of 2p+1).
double build_levels(const stst_problem *h, const std::vector<Term> &terms, const int *ord,
                    std::vector<LevelSpec> &levels) {
  const int d = h->d;
  const int L = d + 1;
  levels.clear();
  // level 0: distinct matrices of mode ord[0]
  std::map<int, int> out0;
  for (const Term &t : terms) {
    int mid = t.m[ord[0]];
    if (!out0.count(mid)) {
      int k = (int)out0.size();
      out0[mid] = k;
    }
  }
  {
    LevelSpec s;
    s.mode = ord[0];
    s.n_in = 1;
    s.n_out = (int)out0.size();
    for (auto &kv : out0) s.apps.push_back({0, kv.first});
    // apps are in map order; output index = map value
    s.coef.assign(s.apps.size(), std::vector<double>(s.n_out, 0.0));
    for (size_t a = 0; a < s.apps.size(); ++a) s.coef[a][out0[s.apps[a].second]] = 1.0;
    levels.push_back(s);
  }
  // each term's current tensor index (output of previous level) and remaining key
  std::vector<int> cur(terms.size());
  for (size_t k = 0; k < terms.size(); ++k) cur[k] = out0[terms[k].m[ord[0]]];
  for (int lev = 1; lev < L; ++lev) {
    const int mode = ord[lev];
    LevelSpec s;
    s.mode = mode;
    s.n_in = (int)levels.back().n_out;
    std::map<std::pair<int, int>, int> appid;      // (input, matrix) -> app
    std::map<std::vector<int>, int> outid;         // remaining matrices -> output
    std::vector<int> tapp(terms.size()), tout(terms.size());
    for (size_t k = 0; k < terms.size(); ++k) {
      std::pair<int, int> key(cur[k], terms[k].m[mode]);
      if (!appid.count(key)) {
        int id = (int)appid.size();
        appid[key] = id;
      }
      tapp[k] = appid[key];
      std::vector<int> rest;
      for (int r = lev + 1; r < L; ++r) rest.push_back(terms[k].m[ord[r]]);
      if (!outid.count(rest)) {
        int id = (int)outid.size();
        outid[rest] = id;
      }
      tout[k] = outid[rest];
    }
    s.n_out = (int)outid.size();
    s.apps.resize(appid.size());
    for (auto &kv : appid) s.apps[kv.second] = kv.first;
    s.coef.assign(s.apps.size(), std::vector<double>(s.n_out, 0.0));
    for (size_t k = 0; k < terms.size(); ++k) {
      double c = (lev == 1) ? terms[k].coef : 1.0;
      if (lev == 1) s.coef[tapp[k]][tout[k]] += c;
      else s.coef[tapp[k]][tout[k]] = 1.0;
    }
    // at level >= 2 several terms share (input, matrix, output); coefficient stays 1
    levels.push_back(s);
    for (size_t k = 0; k < terms.size(); ++k) cur[k] = tout[k];
  }
  if (L == 1) return 0.0;
  double work = 0.0;
  for (const LevelSpec &s : levels) {
    int contrib = 0;
    for (size_t a = 0; a < s.apps.size(); ++a)
      for (int b = 0; b < s.n_out; ++b)
        if (s.coef[a][b] != 0.0) contrib++;
    work += contrib * (2.0 * h->dir[s.mode].p + 1.0);
  }
  return work;
}

int make_plan(stst_problem *h, const std::vector<Term> &terms, bool lift, Plan &plan, int *pool_need) {
  const int d = h->d;
  int ord[STST_MAXD + 1], best[STST_MAXD + 1];
  for (int l = 0; l <= d; ++l) ord[l] = l;
  double best_work = 1e300;
  std::vector<LevelSpec> levels, best_levels;
  do {
    if (lift && ord[0] != 0) continue;
    double w = build_levels(h, terms, ord, levels);
    bool ok = true;
    for (const LevelSpec &s : levels) {
      int contrib = 0;
      for (size_t a = 0; a < s.apps.size(); ++a)
        for (int b = 0; b < s.n_out; ++b)
          if (s.coef[a][b] != 0.0) contrib++;
      if (s.n_in > PASS_MAXIN || s.n_out > PASS_MAXOUT || contrib > PASS_MAXAPP || (int)s.apps.size() > PASS_MAXAPP)
        ok = false;
    }
    if (ok && w < best_work) {
      best_work = w;
      best_levels = levels;
      std::copy(ord, ord + d + 1, best);
    }
  } while (std::next_permutation(ord, ord + d + 1));
  if (best_work > 1e299) return STST_ERR_ARG;
  (void)best;
  // geometry and pointers
  plan.passes.clear();
  long long ext[STST_MAXD + 1];
  for (int l = 0; l <= d; ++l) ext[l] = h->dir[l].n;
  int need = 0;
  for (size_t lev = 0; lev < best_levels.size(); ++lev) {
    const LevelSpec &s = best_levels[lev];
    PassParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.mode = s.mode;
    pp.p = h->dir[s.mode].p;
    pp.n_in = s.n_in;
    pp.n_out = s.n_out;
    pp.n_app = (int)s.apps.size();
    long long inner = 1, outer = 1;
    for (int k = 0; k < s.mode; ++k) inner *= ext[k];
    for (int k = s.mode + 1; k <= d; ++k) outer *= ext[k];
    pp.inner = inner;
    pp.outer = outer;
    pp.n_mode_out = h->dir[s.mode].n;
    pp.n_mode_in = h->dir[s.mode].n;
    pp.row_off = 0;
    bool lift_time = lift && lev == 0;
    if (lift_time) {
      // input: c on the first (removed) time function only; rows 1..n_t of the full time matrices
      pp.n_mode_in = 1;
      pp.row_off = 1;
      // inner = 1 (time is mode 0); outer = N_s
    }
    for (int a = 0; a < pp.n_app; ++a) {
      int mid = s.apps[a].second;
      pp.app_in[a] = s.apps[a].first;
      if (lift_time) {
        const int bw = 2 * h->dir[0].p + 1;
        pp.mat[a] = h->tfull[mid].d + bw;
        pp.mat32[a] = h->tfull32[mid] + bw;
      } else {
        pp.mat[a] = h->mats[s.mode][mid].d;
        pp.mat32[a] = h->mats32[s.mode][mid];
      }
      pp.app_imag[a] = (s.mode == 0 && mid == TM_KA) ? 1 : 0;
      for (int b = 0; b < pp.n_out; ++b) pp.coef[a][b] = s.coef[a][b];
    }
    plan.passes.push_back(pp);
    if (lev + 1 < best_levels.size()) need = std::max(need, s.n_out);
  }
  *pool_need = need;
  return STST_OK;
}

std::vector<Term> base_terms(const stst_problem *h) {
  std::vector<Term> T;
  const int d = h->d;
  const double nu = h->nu;
  auto mk = [&](double c, int tm) {
    Term t;
    t.coef = c;
    t.m[0] = tm;
    for (int l = 1; l <= d; ++l) t.m[l] = SM_M;
    for (int l = d + 1; l <= STST_MAXD; ++l) t.m[l] = 0;
    return t;
  };
  T.push_back(mk(1.0, TM_L));
  for (int l = 1; l <= d; ++l) {
    Term t = mk(nu * nu, TM_M);
    t.m[l] = SM_J;
    T.push_back(t);
    for (int k = l + 1; k <= d; ++k) {
      Term u = mk(2.0 * nu * nu, TM_M);
      u.m[l] = SM_L;
      u.m[k] = SM_L;
      T.push_back(u);
    }
    Term w = mk(nu, TM_KA);
    w.m[l] = SM_L;
    T.push_back(w);
  }
  return T;
}

// c1 * mats[l][i1] + c2 * mats[l][i2] as a new band matrix of direction l; returns its id
int add_combo(stst_problem *h, int l, int i1, double c1, int i2, double c2) {
  const DirInfo &D = h->dir[l];
  BandMat B;
  B.n = D.n;
  B.p = D.p;
  const int nb = B.n * (2 * B.p + 1);
  STST_TRY(alloc((void **)&B.d, sizeof(double) * nb));
  float *f32 = nullptr;
  int s = alloc((void **)&f32, sizeof(float) * nb);
  if (s == STST_OK) s = launch_band_axpby(h->mats[l][i1].d, c1, h->mats[l][i2].d, c2, B.d, f32, nb, h->stream);
  if (s != STST_OK) {
    cudaFree(B.d);
    cudaFree(f32);
    return s;
  }
  h->mats[l].push_back(B);
  h->mats32[l].push_back(f32);
  return (int)h->mats[l].size() - 1;
}

// Kronecker terms that differ in the matrix of a single spatial mode are combined:
// c1 (.. x A x ..) + c2 (.. x B x ..) = (.. x (c1 A + c2 B) x ..). Fewer terms mean fewer band
// applications in every level of the sum-factorised mat-vec. Time matrices are never combined
// (the imaginary advection term and the lifting's unrestricted time columns stay separate).
std::vector<Term> combine_terms(stst_problem *h, std::vector<Term> t) {
  const int d = h->d;
  for (bool found = true; found;) {
    found = false;
    for (size_t i = 0; i < t.size() && !found; ++i)
      for (size_t j = i + 1; j < t.size() && !found; ++j) {
        int diff = -1, ndiff = 0;
        for (int l = 0; l <= d; ++l)
          if (t[i].m[l] != t[j].m[l]) {
            diff = l;
            ndiff++;
          }
        if (ndiff != 1 || diff == 0) continue;
        const int id = add_combo(h, diff, t[i].m[diff], t[i].coef, t[j].m[diff], t[j].coef);
        if (id < 0) return t;
        Term m = t[i];
        m.coef = 1.0;
        m.m[diff] = id;
        t[i] = m;
        t.erase(t.begin() + j);
        found = true;
      }
  }
  return t;
}

std::vector<Term> merge_terms(const std::vector<Term> &in) {
  std::vector<Term> out;
  for (const Term &t : in) {
    bool found = false;
    for (Term &o : out) {
      if (!memcmp(o.m, t.m, sizeof(t.m))) {
        o.coef += t.coef;
        found = true;
        break;
      }
    }
    if (!found) out.push_back(t);
  }
  return out;
}

int free_pool(stst_problem *h) {
  for (void *p : h->pool) cudaFree(p);
  h->pool.clear();
  return STST_OK;
}

// The plans and the solver graphs captured from them hold pointers into the band matrices and the
// intermediate pool. They are dropped whenever those change: run_plan refuses an empty plan
// (STST_ERR_STATE) and the graphs are rebuilt by the next solve.
// the captured solver graphs alone (their kernels or arguments change, the plans stay)
void invalidate_graphs(stst_problem *h) {
  h->pcg_graph_valid = 0;
  if (h->pcg_exec) {
    cudaGraphExecDestroy(h->pcg_exec);
    h->pcg_exec = nullptr;
  }
  h->ir_graph_valid = 0;
  if (h->ir_exec) {
    cudaGraphExecDestroy(h->ir_exec);
    h->ir_exec = nullptr;
  }
}

void invalidate_plans(stst_problem *h) {
  h->sys_plan.passes.clear();
  h->lift_plan.passes.clear();
  h->pcg_graph_valid = 0;
  if (h->pcg_exec) {
    cudaGraphExecDestroy(h->pcg_exec);
    h->pcg_exec = nullptr;
  }
  h->ir_graph_valid = 0;
  if (h->ir_exec) {
    cudaGraphExecDestroy(h->ir_exec);
    h->ir_exec = nullptr;
  }
}

int replan_impl(stst_problem *h, const std::vector<Term> &terms);

int replan(stst_problem *h, const std::vector<Term> &terms) {
  invalidate_plans(h);
  const int s = replan_impl(h, terms);
  if (s != STST_OK) invalidate_plans(h);
  h->sys_plan.geo = h->geo;
  for (Plan *pl : {&h->sys_plan, &h->lift_plan}) {
    pl->fuse = h->no_fuse ? 0 : 1;
    pl->gbar = h->gbar;
    pl->gerr = h->flags + 1;
  }
  return s;
}

int replan_impl(stst_problem *h, const std::vector<Term> &terms) {
  int need1 = 0, need2 = 0;
  STST_TRY(make_plan(h, terms, false, h->sys_plan, &need1));
  // lifting: time matrices are the full ones; same term list (time ids index tfull)
  STST_TRY(make_plan(h, terms, true, h->lift_plan, &need2));
  free_pool(h);
  // pool: two alternating sets of intermediate tensors (even / odd levels)
  int need = std::max(need1, need2);
  const size_t bytes = sizeof(double2) * (size_t)h->N_dof;
  std::vector<void *> even, odd;
  for (int i = 0; i < need; ++i) {
    void *a, *b;
    STST_TRY(alloc(&a, bytes));
    STST_TRY(alloc(&b, bytes));
    even.push_back(a);
    odd.push_back(b);
    h->pool.push_back(a);
    h->pool.push_back(b);
  }
  for (void *q : h->scaled) cudaFree(q);
  h->scaled.clear();
  for (Plan *pl : {&h->sys_plan, &h->lift_plan}) {
    for (size_t lev = 0; lev < pl->passes.size(); ++lev) {
      PassParams &pp = pl->passes[lev];
      // coefficient-scaled copies of the band matrices (coefficient 1 keeps the original)
      const int nb = pp.n_mode_out * (2 * pp.p + 1);
      for (int a = 0; a < pp.n_app; ++a)
        for (int b = 0; b < pp.n_out; ++b) {
          pp.cmat[a][b] = nullptr;
          pp.cmat32[a][b] = nullptr;
          const double c = pp.coef[a][b];
          if (c == 0.0) continue;
          if (c == 1.0) {
            pp.cmat[a][b] = pp.mat[a];
            pp.cmat32[a][b] = pp.mat32[a];
            continue;
          }
          void *m64, *m32;
          STST_TRY(alloc(&m64, sizeof(double) * nb));
          h->scaled.push_back(m64);
          STST_TRY(alloc(&m32, sizeof(float) * nb));
          h->scaled.push_back(m32);
          STST_TRY(launch_scale(pp.mat[a], c, (double *)m64, (float *)m32, nb, h->stream));
          pp.cmat[a][b] = (const double *)m64;
          pp.cmat32[a][b] = (const float *)m32;
        }
      std::vector<void *> &dst = (lev % 2 == 0) ? even : odd;
      std::vector<void *> &src = (lev % 2 == 0) ? odd : even;
      for (int b = 0; b < pp.n_out; ++b) pp.out[b] = (b < (int)dst.size()) ? dst[b] : nullptr;
      if (lev > 0)
        for (int a = 0; a < pp.n_in; ++a) pp.in[a] = src[a];
    }
  }
  return STST_OK;
}

int check(stst_handle h) {
  if (!h || h->magic != STST_MAGIC) return STST_ERR_HANDLE;
  return STST_OK;
}

void destroy_all(stst_problem *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int l = 0; l <= STST_MAXD; ++l) {
    for (auto &b : h->mats[l]) cudaFree(b.d);
    for (auto *f : h->mats32[l]) cudaFree(f);
    cudaFree(h->qpts[l]);
    cudaFree(h->qwts[l]);
    cudaFree(h->tab[l]);
    cudaFree(h->mchol[l]);
    cudaFree(h->U[l]);
    cudaFree(h->U32[l]);
    cudaFree(h->Ubf[l]);
    cudaFree(h->Utf[l]);
    cudaFree(h->lam[l]);
  }
  for (int k = 0; k < 3; ++k) {
    cudaFree(h->tfull[k].d);
    cudaFree(h->tfull32[k]);
  }
  free_geo(h->geo);
  h->geo = nullptr;
  for (double *p : h->pot_bufs) cudaFree(p);
  free_pool(h);
  for (void *q : h->scaled) cudaFree(q);
  cudaFree(h->oa_work);
  cudaFree(h->Hg);
  cudaFree(h->Hd);
  cudaFree(h->Hg32);
  cudaFree(h->Hd32);
  cudaFree(h->Gp32);
  cudaFree(h->Dp32);
  for (int q = 0; q < 2; ++q) {
    cudaFree(h->Tf[q]);
    cudaFree(h->Tb[q]);
  }
  cudaFree(h->flags);
  cudaFree(h->gbar);
  double *ws[] = {h->w_x, h->w_r, h->w_z, h->w_zold, h->w_p, h->w_q, h->w_f, h->w_t1, h->w_t2};
  for (double *w : ws) cudaFree(w);
  float *vs[] = {h->v_d, h->v_r, h->v_z, h->v_p, h->v_q};
  for (float *v : vs) cudaFree(v);
  cudaFree(h->partials);
  cudaFree(h->ctl);
  cudaFree(h->ctl2);
  cudaFree(h->proj_work);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->flags_host) cudaFreeHost(h->flags_host);
  if (h->pcg_exec) cudaGraphExecDestroy(h->pcg_exec);
  if (h->ir_exec) cudaGraphExecDestroy(h->ir_exec);
  if (h->prof) {
    for (cudaEvent_t e : h->prof->pool) cudaEventDestroy(e);
    delete h->prof;
  }
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->magic = 0;
  delete h;
}

int create_impl(stst_problem *h, int d, const int *n_el, const int *p, double T, double nu, int prec_mode,
                int formulation) {
  cudaStream_t st = h->stream;
  for (int l = 0; l <= d; ++l) {
    DirInfo &D = h->dir[l];
    D.p = p[l];
    D.n_el = n_el[l];
    D.nq = p[l] + 2;
    D.m = n_el[l] + p[l];
    D.n = (l == 0) ? D.m - 1 : D.m - 2;
    D.len = (l == 0) ? T : 1.0;
    // time: the least-squares space drops the first function (initial condition), the ultraweak
    // one the last (final condition); space: both ends (Dirichlet)
    D.off = (l == 0 && formulation == STST_FORM_UW) ? 0 : 1;
  }
  h->formulation = formulation;
  h->d = d;
  h->T = T;
  h->nu = nu;
  h->prec_mode = prec_mode;
  h->N_s = 1;
  for (int l = 1; l <= d; ++l) h->N_s *= h->dir[l].n;
  h->N_dof = h->N_s * h->dir[0].n;
  // quadrature and tables
  for (int l = 0; l <= d; ++l) {
    const DirInfo &D = h->dir[l];
    STST_TRY(alloc((void **)&h->qpts[l], sizeof(double) * D.Q()));
    STST_TRY(alloc((void **)&h->qwts[l], sizeof(double) * D.Q()));
    STST_TRY(alloc((void **)&h->tab[l], sizeof(double) * D.Q() * (D.p + 1) * 3));
    STST_TRY(launch_quadrature(D.p, D.n_el, D.len, D.nq, h->qpts[l], h->qwts[l], h->tab[l], st));
  }
  // time matrices (reduced) : ids TM_L, TM_M, TM_KA
  add_band(h, 0, MK_L, nullptr);
  add_band(h, 0, MK_M, nullptr);
  add_band(h, 0, MK_KA, nullptr);
  // full time matrices for the lifting of the initial datum
  {
    const DirInfo &D = h->dir[0];
    int kinds[3] = {MK_L, MK_M, MK_KA};
    for (int k = 0; k < 3; ++k) {
      BandMat &B = h->tfull[k];
      B.n = D.m;
      B.p = D.p;
      STST_TRY(alloc((void **)&B.d, sizeof(double) * B.n * (2 * B.p + 1)));
      STST_TRY(launch_assemble_band(kinds[k], D.p, D.n_el, D.len, D.nq, 0, D.m, D.m, nullptr, B.d, st));
      STST_TRY(alloc((void **)&h->tfull32[k], sizeof(float) * B.n * (2 * B.p + 1)));
      STST_TRY(launch_to_f32(B.d, h->tfull32[k], (long long)B.n * (2 * B.p + 1), st));
    }
  }
  STST_CUDA(cudaMalloc(&h->flags, sizeof(int) * 4));
  STST_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int) * 4, st));
  STST_CUDA(cudaMalloc(&h->gbar, sizeof(unsigned) * 2));
  STST_CUDA(cudaMemsetAsync(h->gbar, 0, sizeof(unsigned) * 2, st));
  for (int l = 1; l <= d; ++l) {
    add_band(h, l, MK_M, nullptr);    // SM_M
    add_band(h, l, MK_L, nullptr);    // SM_L
    add_band(h, l, MK_J, nullptr);    // SM_J
    add_band(h, l, MK_K2S, nullptr);  // SM_K2S (unit weight)
    const DirInfo &D = h->dir[l];
    STST_TRY(alloc((void **)&h->mchol[l], sizeof(double) * D.n * (D.p + 1)));
    STST_TRY(launch_mass_cholesky(h->mats[l][SM_M], h->mchol[l], h->flags, st));
    STST_TRY(alloc((void **)&h->U[l], sizeof(double) * D.n * D.n));
    STST_TRY(alloc((void **)&h->U32[l], sizeof(float) * D.n * D.n));
    STST_TRY(alloc((void **)&h->Ubf[l], sizeof(__nv_bfloat16) * 4 * pad16(D.n) * pad16(D.n)));
    STST_TRY(alloc((void **)&h->Utf[l], sizeof(float) * tf32_planes_floats(D.n)));
    STST_TRY(alloc((void **)&h->lam[l], sizeof(double) * D.n));
  }
  int nmax = 1;
  for (int l = 1; l <= d; ++l) nmax = std::max(nmax, h->dir[l].n);
  STST_TRY(alloc((void **)&h->oa_work, sizeof(double) * 6 * nmax * nmax));
  const long long nt = h->dir[0].n, Pt = h->dir[0].p;
  STST_TRY(alloc(&h->Hg, sizeof(double2) * nt * Pt * h->N_s));
  STST_TRY(alloc((void **)&h->Hd, sizeof(double) * nt * h->N_s));
  STST_TRY(alloc(&h->Hg32, sizeof(float2) * nt * Pt * h->N_s));
  STST_TRY(alloc((void **)&h->Hd32, sizeof(float) * nt * h->N_s));
  if (prec_mode == STST_PREC_FP32 && (pencil_fits(h, 1) || pencil_fits(h, 2))) {
    STST_TRY(alloc(&h->Gp32, sizeof(float2) * nt * Pt * h->N_s));
    STST_TRY(alloc((void **)&h->Dp32, sizeof(float) * nt * h->N_s));
  }
  for (int q = 0; q < 2; ++q) {  // transfer matrices of the segmented time solves (FP64 ones in FP64 mode)
    h->ts_S[q] = 0;
    if (q == 1 && prec_mode != STST_PREC_FP64) continue;
    ts_segments((int)nt, (int)Pt, q ? sizeof(double) : sizeof(float), &h->ts_S[q], &h->ts_L[q]);
    if (h->ts_S[q] < 2) continue;
    const size_t cnt = (size_t)h->ts_S[q] * Pt * Pt * h->N_s * (q ? sizeof(double2) : sizeof(float2));
    STST_TRY(alloc(&h->Tf[q], cnt));
    STST_TRY(alloc(&h->Tb[q], cnt));
  }
  const size_t vb = sizeof(double2) * (size_t)h->N_dof;
  double **ws[] = {&h->w_x, &h->w_r, &h->w_z, &h->w_zold, &h->w_p, &h->w_q, &h->w_f, &h->w_t1, &h->w_t2};
  for (double **w : ws) STST_TRY(alloc((void **)w, vb));
  STST_TRY(alloc((void **)&h->partials, sizeof(double) * PS_COUNT * STST_MAXPART));
  STST_TRY(alloc((void **)&h->ctl, sizeof(PcgCtl)));
  STST_TRY(alloc((void **)&h->ctl2, sizeof(PcgCtl)));
  float **vs[] = {&h->v_d, &h->v_r, &h->v_z, &h->v_p, &h->v_q};
  for (float **v : vs) STST_TRY(alloc((void **)v, sizeof(float2) * (size_t)h->N_dof));
  {
    cudaError_t e = cudaMallocHost(&h->ctl_host, 2 * sizeof(PcgCtl));
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      return STST_ERR_OOM;
    }
    e = cudaMallocHost(&h->flags_host, 4 * sizeof(int));
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      return STST_ERR_OOM;
    }
  }
  // projection workspace: largest partially contracted spatial tensor
  {
    long long mx = h->N_s;
    for (int l = 1; l <= d; ++l) {
      long long s = 1;
      for (int k = 1; k <= d; ++k) s *= (k <= l) ? h->dir[k].n : h->dir[k].Q();
      mx = std::max(mx, s);
    }
    h->proj_work_bytes = 3 * sizeof(double2) * (size_t)mx;
    STST_TRY(alloc((void **)&h->proj_work, h->proj_work_bytes));
  }
  h->pot_rank = 0;
  STST_TRY(replan(h, base_terms(h)));
  STST_CUDA(cudaStreamSynchronize(st));
  int fl[4];
  STST_CUDA(cudaMemcpy(fl, h->flags, sizeof(fl), cudaMemcpyDeviceToHost));
  if (fl[0]) return STST_NOT_HPD;
  return STST_OK;
}

}  // namespace

// for the mapped-domain operator (geometry.cu): its setup changes the kernels the solver graphs hold
void invalidate_solver_graphs(stst_problem *h) { invalidate_graphs(h); }

extern "C" {

const char *stst_strerror(int s) {
  switch (s) {
    case STST_OK: return "ok";
    case STST_NOT_CONVERGED: return "not converged within maxit";
    case STST_BREAKDOWN: return "CG breakdown (<p,Ap> <= 0 or non-finite)";
    case STST_NOT_HPD: return "factorization met a non-positive pivot";
    case STST_TIMEOUT: return "a bounded device wait expired";
    case STST_ERR_ARG: return "invalid argument";
    case STST_ERR_HANDLE: return "invalid handle";
    case STST_ERR_OOM: return "device allocation failed";
    case STST_ERR_CUDA: return "CUDA runtime error";
    case STST_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

int stst_create(stst_handle *out, int d, const int *n_el, const int *p, double T, double nu, int prec_mode,
                void *stream) {
  return stst_create2(out, d, n_el, p, T, nu, prec_mode, STST_FORM_LS, stream);
}

int stst_create2(stst_handle *out, int d, const int *n_el, const int *p, double T, double nu, int prec_mode,
                 int formulation, void *stream) {
  if (!out || !n_el || !p) return STST_ERR_ARG;
  if (formulation != STST_FORM_LS && formulation != STST_FORM_UW) return STST_ERR_ARG;
  *out = nullptr;
  if (d < 1 || d > STST_MAXD) return STST_ERR_ARG;
  if (!(T > 0.0) || !(nu > 0.0) || !std::isfinite(T) || !std::isfinite(nu)) return STST_ERR_ARG;
  if (prec_mode < STST_PREC_FP64 || prec_mode > STST_PREC_BF16) return STST_ERR_ARG;
  if (p[0] < 1 || p[0] > STST_MAXP || n_el[0] < 1 || n_el[0] > (1 << 20)) return STST_ERR_ARG;
  for (int l = 1; l <= d; ++l) {
    if (p[l] < 2 || p[l] > STST_MAXP || n_el[l] < 1) return STST_ERR_ARG;
    int n = n_el[l] + p[l] - 2;
    if (n < 1 || n > STST_MAXN_SPACE) return STST_ERR_ARG;
  }
  stst_problem *h = new (std::nothrow) stst_problem();  // value-initialized: every scalar member is zero
  if (!h) return STST_ERR_OOM;
  h->magic = STST_MAGIC;
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {
    // CUDA graphs cannot be captured on the legacy default stream. A blocking stream still
    // orders implicitly with work the caller puts on the legacy default stream.
    cudaError_t e = cudaStreamCreate(&h->stream);
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      delete h;
      return STST_ERR_CUDA;
    }
    h->own_stream = 1;
  }
  for (int l = 1; l <= d; ++l) h->mp_cfg[l] = modeprod_default(n_el[l] + p[l] - 2);
  int s = create_impl(h, d, n_el, p, T, nu, prec_mode, formulation);
  if (s != STST_OK) {
    destroy_all(h);
    return s;
  }
  *out = h;
  return STST_OK;
}

int stst_destroy(stst_handle h) {
  STST_TRY(check(h));
  destroy_all(h);
  return STST_OK;
}

int stst_sizes(stst_handle h, long long *n_dof, int *n) {
  STST_TRY(check(h));
  if (n_dof) *n_dof = h->N_dof;
  if (n)
    for (int l = 0; l <= h->d; ++l) n[l] = h->dir[l].n;
  return STST_OK;
}

int stst_quadrature_points(stst_handle h, int dir, double *pts) {
  STST_TRY(check(h));
  if (dir < 0 || dir > h->d || !pts) return STST_ERR_ARG;
  STST_CUDA(cudaMemcpyAsync(pts, h->qpts[dir], sizeof(double) * h->dir[dir].Q(), cudaMemcpyDeviceToDevice,
                            h->stream));
  return STST_OK;
}

int stst_assemble_1d(int p, int n_el, double length, int bc, const double *weight, double *M, double *L, double *J,
                     double *K, double *K2, int *n_out, void *stream) {
  if (p < 1 || p > STST_MAXP || n_el < 1 || !(length > 0.0) || bc < 0 || bc > 2) return STST_ERR_ARG;
  int m = n_el + p;
  int n = m - bc;
  int off = bc > 0 ? 1 : 0;
  if (n < 1) return STST_ERR_ARG;
  if (n_out) *n_out = n;
  cudaStream_t st = (cudaStream_t)stream;
  double *outs[5] = {M, L, J, K, K2};
  int kinds[5] = {MK_M, MK_L, MK_J, MK_K, MK_K2};
  for (int k = 0; k < 5; ++k)
    if (outs[k]) STST_TRY(launch_assemble_band(kinds[k], p, n_el, length, p + 2, off, n, n, weight, outs[k], st));
  return STST_OK;
}

// Additive potential V = sum_l v_l(x_l) (each factor differs from 1 in one direction only, one factor per
// direction): the operator is i d_t + sum_l H_l with H_l = -nu d_ll + v_l, so the least-squares matrix
// (Sec. 4.3, Eq. syst_mat with the potential's terms) is
//   L_t (x) M..M + sum_l KA (x) G_l + sum_l M_t (x) A_l + 2 sum_{l<k} M_t (x) G_l (x) G_k
// (each G_l / A_l at position l, M elsewhere), G_l = nu L_l + M_{v_l} (the Galerkin matrix of H_l) and
// A_l = nu^2 J_l + M_{v_l^2} - nu (K2_{v_l} + K2_{v_l}^T). The cross terms 2 nu^2 L (x) L + 2 M_v (x) M_v
// - nu M_v (x) K2S - nu K2S (x) M_v of the general expansion are 2 G_l (x) G_k because K2 + K2^T = -2 L
// for spatial functions that vanish on the boundary (integration by parts). The same matrix in fewer
// Kronecker terms: the mat-vec needs as many band applications as with V = 0.
static int additive_terms(stst_problem *h, int rank, const int *dir_of, const int (*wm)[3], const int (*wk)[3],
                          const int (*pm)[3][3], std::vector<Term> &T) {
  const int d = h->d;
  const double nu = h->nu;
  int gm[STST_MAXD + 1], am[STST_MAXD + 1];
  double gc[STST_MAXD + 1], ac[STST_MAXD + 1];
  for (int l = 1; l <= d; ++l) {
    int r = -1;
    for (int q = 0; q < rank; ++q)
      if (dir_of[q] == l) r = q;
    if (r < 0) {
      gm[l] = SM_L, gc[l] = nu;
      am[l] = SM_J, ac[l] = nu * nu;
      const int g = add_combo(h, l, SM_L, nu, SM_M, 0.0);  // nu L_l as a matrix of its own for the FD setup
      if (g < 0) return g;
      h->g_mat[l] = g;
      continue;
    }
    const int g = add_combo(h, l, SM_L, nu, wm[l][r], 1.0);
    if (g < 0) return g;
    const int a1 = add_combo(h, l, SM_J, nu * nu, pm[l][r][r], 1.0);
    if (a1 < 0) return a1;
    const int a = add_combo(h, l, a1, 1.0, wk[l][r], -nu);
    if (a < 0) return a;
    gm[l] = g, gc[l] = 1.0;
    am[l] = a, ac[l] = 1.0;
    h->g_mat[l] = g;
  }
  h->g_valid = 1;
  auto mk = [&](double c, int tm) {
    Term t;
    t.coef = c;
    t.m[0] = tm;
    for (int l = 1; l <= STST_MAXD; ++l) t.m[l] = (l <= d) ? SM_M : 0;
    return t;
  };
  T.clear();
  T.push_back(mk(1.0, TM_L));
  for (int l = 1; l <= d; ++l) {
    Term w = mk(gc[l], TM_KA);
    w.m[l] = gm[l];
    T.push_back(w);
    Term a = mk(ac[l], TM_M);
    a.m[l] = am[l];
    T.push_back(a);
    for (int k = l + 1; k <= d; ++k) {
      Term c = mk(2.0 * gc[l] * gc[k], TM_M);
      c.m[l] = gm[l];
      c.m[k] = gm[k];
      T.push_back(c);
    }
  }
  return STST_OK;
}

// Removes the potential: its band matrices (ids beyond SM_K2S, including the combined ones) and weight
// buffers are freed, so the plans that point at them are dropped as well until the next replan.
static void drop_potential(stst_problem *h) {
  invalidate_plans(h);
  for (int l = 1; l <= h->d; ++l) {
    while ((int)h->mats[l].size() > SM_K2S + 1) {
      cudaFree(h->mats[l].back().d);
      cudaFree(h->mats32[l].back());
      h->mats[l].pop_back();
      h->mats32[l].pop_back();
    }
  }
  for (double *p : h->pot_bufs) cudaFree(p);
  h->pot_bufs.clear();
  h->pot_rank = 0;
  h->g_valid = 0;
  if (h->prec_op == 1) h->fd_ready = 0;  // the potential-aware factors depend on V
}

static int set_potential_impl(stst_problem *h, int rank, const double *v_qp, const std::vector<double> &host);

int stst_set_potential(stst_handle h, int rank, const double *v_qp) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (rank < 0 || rank > 3 || (rank > 0 && !v_qp)) return STST_ERR_ARG;
  if (h->geo && rank > 0) return STST_ERR_STATE;  // the mapped-domain operator has no potential terms
  // the samples are read and checked before anything of the handle changes: a rejected potential
  // leaves the previous operator in place
  std::vector<double> host;
  if (rank > 0) {
    int stride = 0;
    for (int l = 1; l <= h->d; ++l) stride += h->dir[l].Q();
    host.resize((size_t)stride * rank);
    STST_CUDA(cudaStreamSynchronize(h->stream));
    STST_CUDA(cudaMemcpy(host.data(), v_qp, sizeof(double) * host.size(), cudaMemcpyDeviceToHost));
    for (double v : host)
      if (!std::isfinite(v)) return STST_ERR_ARG;
  }
  const int s = set_potential_impl(h, rank, v_qp, host);
  if (s != STST_OK) {
    // a failure part-way (allocation, launch) leaves the V = 0 operator; if even that cannot be planned,
    // every call that needs the mat-vec returns STST_ERR_STATE
    drop_potential(h);
    replan(h, combine_terms(h, merge_terms(base_terms(h))));
    cudaStreamSynchronize(h->stream);
  }
  return s;
}

static int set_potential_impl(stst_problem *h, int rank, const double *v_qp, const std::vector<double> &host) {
  cudaStream_t st = h->stream;
  const int d = h->d;
  drop_potential(h);
  std::vector<Term> terms = base_terms(h);
  if (rank > 0) {
    int stride = 0;
    for (int l = 1; l <= d; ++l) stride += h->dir[l].Q();
    double *vcopy;
    STST_TRY(alloc((void **)&vcopy, sizeof(double) * stride * rank));
    h->pot_bufs.push_back(vcopy);
    STST_CUDA(cudaMemcpyAsync(vcopy, v_qp, sizeof(double) * stride * rank, cudaMemcpyDeviceToDevice, st));
    // weight registry per direction: key = list of factor ids (sorted) -> (M id, K2S id)
    // factor id f in [0, rank): v_{f,l}; "one" if the samples are identically 1.
    int wm[STST_MAXD + 1][3], wk[STST_MAXD + 1][3];
    int pm[STST_MAXD + 1][3][3];
    bool onef[STST_MAXD + 1][3];
    int off = 0;
    for (int l = 1; l <= d; ++l) {
      const int Ql = h->dir[l].Q();
      int canon[3];
      bool one[3];
      for (int r = 0; r < rank; ++r) {
        const double *a = host.data() + (size_t)r * stride + off;
        one[r] = true;
        for (int q = 0; q < Ql; ++q)
          if (a[q] != 1.0) { one[r] = false; break; }
        canon[r] = r;
        for (int s = 0; s < r; ++s) {
          const double *b = host.data() + (size_t)s * stride + off;
          if (!memcmp(a, b, sizeof(double) * Ql)) { canon[r] = canon[s]; break; }
        }
      }
      for (int r = 0; r < rank; ++r) onef[l][r] = one[r];
      for (int r = 0; r < rank; ++r) {
        if (one[r]) { wm[l][r] = SM_M; wk[l][r] = SM_K2S; continue; }
        if (canon[r] != r) { wm[l][r] = wm[l][canon[r]]; wk[l][r] = wk[l][canon[r]]; continue; }
        const double *w = vcopy + (size_t)r * stride + off;
        wm[l][r] = add_band(h, l, MK_M, w);
        if (wm[l][r] < 0) return wm[l][r];
        wk[l][r] = add_band(h, l, MK_K2S, w);
        if (wk[l][r] < 0) return wk[l][r];
      }
      for (int r = 0; r < rank; ++r)
        for (int s = 0; s < rank; ++s) {
          if (one[r]) { pm[l][r][s] = wm[l][s]; continue; }
          if (one[s]) { pm[l][r][s] = wm[l][r]; continue; }
          if (s < r) { pm[l][r][s] = pm[l][s][r]; continue; }
          // product weight
          double *wp;
          STST_TRY(alloc((void **)&wp, sizeof(double) * Ql));
          h->pot_bufs.push_back(wp);
          STST_TRY(launch_weight_product(vcopy + (size_t)r * stride + off, vcopy + (size_t)s * stride + off, wp, Ql,
                                         st));
          pm[l][r][s] = add_band(h, l, MK_M, wp);
          if (pm[l][r][s] < 0) return pm[l][r][s];
        }
      off += Ql;
    }
    // which direction each factor lives in, if every factor is 1 in all directions but one
    int dir_of[3] = {-1, -1, -1};
    bool additive = true, taken[STST_MAXD + 1] = {};
    for (int r = 0; r < rank && additive; ++r) {
      for (int l = 1; l <= d; ++l)
        if (!onef[l][r]) {
          if (dir_of[r] >= 0) additive = false;
          dir_of[r] = l;
        }
      if (dir_of[r] < 0 || taken[dir_of[r]]) additive = false;
      else taken[dir_of[r]] = true;
    }
    if (additive) {
      STST_TRY(additive_terms(h, rank, dir_of, wm, wk, pm, terms));
      // directions whose G_l are equal (same degree and mesh, no factor in either or bitwise equal factor
      // samples) share one eigendecomposition in the potential-aware setup
      int offs[STST_MAXD + 2] = {0};
      for (int l = 1; l <= d; ++l) offs[l + 1] = offs[l] + h->dir[l].Q();
      for (int l = 1; l <= d; ++l) {
        h->g_share[l] = l;
        int rl = -1;
        for (int q = 0; q < rank; ++q)
          if (dir_of[q] == l) rl = q;
        for (int k = 1; k < l && h->g_share[l] == l; ++k) {
          if (h->dir[k].p != h->dir[l].p || h->dir[k].n_el != h->dir[l].n_el) continue;
          int rk = -1;
          for (int q = 0; q < rank; ++q)
            if (dir_of[q] == k) rk = q;
          if ((rk < 0) != (rl < 0)) continue;
          const size_t Q = (size_t)h->dir[l].Q();
          if (rl >= 0 && memcmp(host.data() + (size_t)rk * stride + offs[k], host.data() + (size_t)rl * stride + offs[l],
                                sizeof(double) * Q) != 0)
            continue;
          h->g_share[l] = h->g_share[k];
        }
      }
      h->pot_rank = rank;
      STST_TRY(replan(h, terms));
      STST_CUDA(cudaStreamSynchronize(st));
      return STST_OK;
    }
    for (int r = 0; r < rank; ++r) {
      for (int s = 0; s < rank; ++s) {
        Term t;
        t.coef = 1.0;
        t.m[0] = TM_M;
        for (int l = 1; l <= STST_MAXD; ++l) t.m[l] = (l <= d) ? pm[l][r][s] : 0;
        terms.push_back(t);
      }
      Term w;
      w.coef = 1.0;
      w.m[0] = TM_KA;
      for (int l = 1; l <= STST_MAXD; ++l) w.m[l] = (l <= d) ? wm[l][r] : 0;
      terms.push_back(w);
      for (int l = 1; l <= d; ++l) {
        Term k;
        k.coef = -h->nu;
        k.m[0] = TM_M;
        for (int q = 1; q <= STST_MAXD; ++q) k.m[q] = (q <= d) ? wm[q][r] : 0;
        k.m[l] = wk[l][r];
        terms.push_back(k);
      }
    }
    h->pot_rank = rank;
  }
  STST_TRY(replan(h, combine_terms(h, merge_terms(terms))));
  STST_CUDA(cudaStreamSynchronize(st));
  return STST_OK;
}

int stst_build_fd(stst_handle h) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (h->prec_op == 1 && h->pot_rank > 0 && !h->g_valid) return STST_ERR_STATE;  // P_V needs a sum of one-direction factors
  STST_TRY(fd_setup(h));
  return tune_modeprod(h);
}

const char *stst_last_cuda_error(void) {
  static thread_local char buf[160];
  snprintf(buf, sizeof(buf), "%s: %s", cudaGetErrorName(stst_last_cuda), cudaGetErrorString(stst_last_cuda));
  return buf;
}

int stst_set_autotune(int mode) {
  const int rpt = mode / 10, cpt = mode % 10;
  if (mode != 0 && mode != 1 && mode != 132 && !(rpt >= 1 && rpt <= 4 && (cpt == 2 || cpt == 4))) return STST_ERR_ARG;
  g_tune_enabled = mode;
  return STST_OK;
}

int stst_set_fused_transforms(int mode) {
  if (mode < 0 || (mode > 2 && (mode < 11 || mode > 14))) return STST_ERR_ARG;
  g_fd2d_mode = mode;
  return STST_OK;
}

int stst_fused_transforms_info(stst_handle h, int *fused) {
  STST_TRY(check(h));
  if (fused) *fused = h->fd2d;
  return STST_OK;
}

int stst_fused_transforms_split(stst_handle h, int *forward, int *backward) {
  STST_TRY(check(h));
  if (forward) *forward = h->fd2d;
  if (backward) *backward = h->fd2d ? h->fd2d_b : 0;
  return STST_OK;
}

int stst_set_pencil(int mode) {
  if (mode < 0 || mode > 3) return STST_ERR_ARG;
  g_pencil_mode = mode;
  return STST_OK;
}

int stst_pencil_info(stst_handle h, int *ctas_per_pencil) {
  STST_TRY(check(h));
  if (ctas_per_pencil) *ctas_per_pencil = h->pencil;
  return STST_OK;
}

extern int g_tf32_mode;

int stst_set_fused_matvec(int mode) {
  if (mode < 0 || mode > 1) return STST_ERR_ARG;
  g_fused_matvec = mode;
  return STST_OK;
}

int stst_set_tensor_products(int mode) {
  if (mode < 0 || mode > 2) return STST_ERR_ARG;
  g_tf32_mode = mode;
  return STST_OK;
}

int stst_tensor_products_info(stst_handle h, int *dirs) {
  STST_TRY(check(h));
  int mask = 0;
  if (h->prec_mode == STST_PREC_FP32)
    for (int l = 1; l <= h->d; ++l)
      if (h->mp_cfg[l].tc) mask |= 1 << l;
  if (dirs) *dirs = mask;
  return STST_OK;
}

int stst_set_time_solver(int mode) {
  if (mode < 0 || mode > 2) return STST_ERR_ARG;
  g_ts_mode = mode;
  return STST_OK;
}

int stst_time_solver_info(stst_handle h, int precision, int *segments, int *segment_len, int *segmented) {
  STST_TRY(check(h));
  if (precision != 0 && precision != 1) return STST_ERR_ARG;
  const int q = precision == 0 ? 1 : 0;  // STST_PREC_FP64 uses the FP64 factors
  if (segments) *segments = h->ts_S[q];
  if (segment_len) *segment_len = h->ts_L[q];
  if (segmented) *segmented = h->ts_seg[q];
  return STST_OK;
}

int stst_tile_info(stst_handle h, int dir, int *cols_per_cta, int *rows_per_cta, double *us) {
  STST_TRY(check(h));
  if (dir < 1 || dir > h->d) return STST_ERR_ARG;
  if (cols_per_cta) *cols_per_cta = 8 * h->mp_cfg[dir].cpt;
  if (rows_per_cta) *rows_per_cta = 32 * h->mp_cfg[dir].rpt;
  if (us) *us = h->mp_us[dir];
  return STST_OK;
}

int stst_apply_sys(stst_handle h, const double *x, double *y) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (!x || !y || x == y) return STST_ERR_ARG;
  return run_plan(h->sys_plan, x, y, 0, 0, nullptr, nullptr, nullptr, nullptr, h->stream);
}

int stst_apply_prec(stst_handle h, const double *r, double *s) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (!r || !s) return STST_ERR_ARG;
  if (!h->fd_ready) return STST_ERR_STATE;
  int prec = h->prec_mode;  // STST_PREC_* equals fd_apply's precision code
  return fd_apply(h, r, s, prec, EpiDot(), nullptr, h->w_t1, h->w_t2);
}

int stst_rhs(stst_handle h, const double *f_qp, const double *u0_qp, double *rhs, double *c0) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (!rhs) return STST_ERR_ARG;
  if (h->geo) return STST_ERR_STATE;  // parametric integrals: the caller assembles a mapped-domain load vector
  return rhs_compute(h, f_qp, u0_qp, rhs, c0);
}

int stst_rhs_lift(stst_handle h, const double *f_qp, const double *u_qp, double *rhs, double *xd) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (h->geo) return STST_ERR_STATE;
  return rhs_lift_compute(h, f_qp, u_qp, rhs, xd);
}

int stst_pcg_solve(stst_handle h, const double *rhs, double *x, double tol, int maxit, int *iters, double *relres) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (!rhs || !x || !(tol >= 0.0) || maxit < 0) return STST_ERR_ARG;
  if (!h->fd_ready) return STST_ERR_STATE;
  return pcg_run(h, rhs, x, tol, maxit, iters, relres);
}

int stst_ir_solve(stst_handle h, const double *rhs, double *x, double tol, int maxit, double inner_tol,
                  int inner_maxit, int *iters, int *outer, double *relres) {
  STST_TRY(check(h));
  ApiScope scope(h);
  if (!rhs || !x || !(tol >= 0.0) || maxit < 0 || !(inner_tol > 0.0) || inner_maxit < 1) return STST_ERR_ARG;
  if (!h->fd_ready) return STST_ERR_STATE;
  return ir_run(h, rhs, x, tol, maxit, inner_tol, inner_maxit, iters, outer, relres);
}

int stst_profile(stst_handle h, int enable) {
  STST_TRY(check(h));
  if (!h->prof) h->prof = new (std::nothrow) Profiler();
  if (!h->prof) return STST_ERR_OOM;
  prof_flush(h->prof);
  if (enable) {
    h->prof->names.clear();
    h->prof->total_ms.clear();
    h->prof->count.clear();
  }
  h->prof_on = enable ? 1 : 0;
  return STST_OK;
}

int stst_set_prec_operator(stst_handle h, int op) {
  STST_TRY(check(h));
  if (op != 0 && op != 1) return STST_ERR_ARG;
  if (op == 1 && h->pot_rank > 0 && !h->g_valid) return STST_ERR_ARG;
  if (op != h->prec_op) h->fd_ready = 0;
  h->prec_op = op;
  return STST_OK;
}

int stst_pcg_graph_info(stst_handle h, int *kernels_per_body, int *iterations_per_body) {
  STST_TRY(check(h));
  if (!h->pcg_graph_valid) return STST_ERR_STATE;
  if (kernels_per_body) *kernels_per_body = h->pcg_body_kernels;
  if (iterations_per_body) *iterations_per_body = 2;
  return STST_OK;
}

int stst_plan_info(stst_handle h, int *n_passes, int *band_apps, double *flops_per_dof) {
  STST_TRY(check(h));
  int apps = 0;
  double flops = 0.0;
  for (const PassParams &pp : h->sys_plan.passes) {
    for (int a = 0; a < pp.n_app; ++a)
      for (int b = 0; b < pp.n_out; ++b)
        if (pp.coef[a][b] != 0.0) {
          apps++;
          flops += 4.0 * (2 * pp.p + 1);
        }
  }
  if (n_passes) *n_passes = (int)h->sys_plan.passes.size();
  if (band_apps) *band_apps = apps;
  if (flops_per_dof) *flops_per_dof = flops;
  return STST_OK;
}

int stst_profile_read(stst_handle h, int idx, char *name, int name_len, long long *count, double *total_ms) {
  STST_TRY(check(h));
  if (h->prof) prof_flush(h->prof);
  if (!h->prof || idx < 0 || idx >= (int)h->prof->names.size()) return STST_ERR_ARG;
  if (name && name_len > 0) {
    const std::string &nm = h->prof->names[idx];
    size_t n = std::min((size_t)name_len - 1, nm.size());
    memcpy(name, nm.data(), n);
    name[n] = 0;
  }
  if (count) *count = h->prof->count[idx];
  if (total_ms) *total_ms = h->prof->total_ms[idx];
  return STST_OK;
}

}  // extern "C"
