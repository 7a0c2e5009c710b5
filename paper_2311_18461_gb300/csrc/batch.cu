// Batched solves: many independent problems (different meshes, degrees, potentials, right-hand
// sides) solved by ONE launch of one CUDA graph. Each problem is an independent branch:
//   [parameters -> control block] [copy rhs, x in] [preconditioner setup] [PCG init]
//   -> WHILE(condition) { one PCG iteration }  -> [copy x out, record iterations / residual / status]
// Branches share nothing, so the GPU runs them concurrently; the loop of each branch ends after at
// most maxit bodies (its control kernel clears the condition), so the graph always terminates.
#include "common.cuh"
#include <new>
#include <vector>

struct BatchParams {
  double tol2;
  int maxit;
  int pad;
};

struct BatchResult {
  int iters, status, setup_flags, pad;
  double relres;
};

struct stst_batch_s {
  int magic;
  int count;
  std::vector<stst_problem *> hs;
  cudaStream_t stream;
  int own_stream;
  BatchParams *params;       // device
  BatchResult *results;      // device
  BatchResult *results_host; // pinned
  cudaGraphExec_t exec;
};

#define STST_BATCH_MAGIC 0x42415443

__global__ void k_batch_ctl(PcgCtl *ctl, const BatchParams *bp, int flexible) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->tol2 = bp->tol2;
    ctl->maxit = bp->maxit;
    ctl->flexible = flexible;
    ctl->it = 0;
    ctl->done = 0;
    ctl->status = STST_OK;
    ctl->x0_zero = 1;  // cleared by pcg_init if the initial guess has a nonzero entry
  }
}

__global__ void k_batch_result(const PcgCtl *ctl, const int *flags, BatchResult *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out->iters = ctl->it;
    out->relres = ctl->ff > 0.0 ? sqrt(ctl->rr / ctl->ff) : 0.0;
    int st = ctl->status;
    if (st == STST_OK && !ctl->done) st = STST_NOT_CONVERGED;
    out->setup_flags = flags[0] | flags[1];
    if (flags[0] & 3) st = STST_NOT_HPD;
    if (flags[1] & 4) st = STST_TIMEOUT;
    out->status = st;
  }
}

static int capture_into(cudaStream_t s, cudaGraph_t g) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  return STST_OK;
}

static int end_capture(cudaStream_t s) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  return STST_OK;
}

// One branch of the batch graph for problem i.
static int add_branch(stst_batch_s *b, cudaGraph_t G, int i, const double *rhs, double *x) {
  stst_problem *h = b->hs[i];
  cudaStream_t st = h->stream;
  const size_t bytes = sizeof(double2) * (size_t)h->N_dof;
  const int flexible = h->prec_mode != STST_PREC_FP64;
  // pre: parameters, copies, setup, init
  cudaGraph_t pre;
  STST_CUDA(cudaGraphCreate(&pre, 0));
  STST_TRY(capture_into(st, pre));
  int s = STST_OK;
  k_batch_ctl<<<1, 32, 0, st>>>(h->ctl, b->params, flexible);
  if (cudaMemcpyAsync(h->w_f, rhs, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) s = STST_ERR_CUDA;
  if (cudaMemcpyAsync(h->w_x, x, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) s = STST_ERR_CUDA;
  if (s == STST_OK) s = fd_setup_launch(h);
  if (s == STST_OK) s = pcg_init(h);
  int s2 = end_capture(st);
  if (s != STST_OK || s2 != STST_OK) {
    cudaGraphDestroy(pre);
    return s != STST_OK ? s : s2;
  }
  cudaGraphNode_t n_pre;
  cudaError_t e = cudaGraphAddChildGraphNode(&n_pre, G, nullptr, 0, pre);
  cudaGraphDestroy(pre);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  // loop: WHILE node depending on the pre part
  cudaGraphConditionalHandle cond;
  STST_CUDA(cudaGraphConditionalHandleCreate(&cond, G, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t n_loop;
  STST_CUDA(cudaGraphAddNode(&n_loop, G, &n_pre, nullptr, 1, &cp));
  STST_TRY(capture_into(st, cp.conditional.phGraph_out[0]));
  s = pcg_body(h, cond, 1);
  if (s == STST_OK) s = pcg_body(h, cond, 1);  // two iterations per body, as in the single-problem graph
  s2 = end_capture(st);
  if (s != STST_OK) return s;
  if (s2 != STST_OK) return s2;
  // post: copy the solution out, record the outcome
  cudaGraph_t post;
  STST_CUDA(cudaGraphCreate(&post, 0));
  STST_TRY(capture_into(st, post));
  if (cudaMemcpyAsync(x, h->w_x, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) s = STST_ERR_CUDA;
  k_batch_result<<<1, 32, 0, st>>>(h->ctl, h->flags, b->results + i);
  s2 = end_capture(st);
  if (s != STST_OK || s2 != STST_OK) {
    cudaGraphDestroy(post);
    return s != STST_OK ? s : s2;
  }
  cudaGraphNode_t n_post;
  e = cudaGraphAddChildGraphNode(&n_post, G, &n_loop, 1, post);
  cudaGraphDestroy(post);
  if (e != cudaSuccess) {
    stst_last_cuda = e;
    return STST_ERR_CUDA;
  }
  return STST_OK;
}

static void batch_free(stst_batch_s *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->params);
  cudaFree(b->results);
  if (b->results_host) cudaFreeHost(b->results_host);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->magic = 0;
  delete b;
}

extern "C" int stst_batch_create(stst_batch *out, int count, const stst_handle *handles, const double *const *rhs,
                                 double *const *x, void *stream) {
  if (!out || count < 1 || !handles || !rhs || !x) return STST_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!handles[i] || handles[i]->magic != STST_MAGIC) return STST_ERR_HANDLE;
    if (!rhs[i] || !x[i]) return STST_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return STST_ERR_ARG;  // one branch per handle (buffers are per handle)
    if (handles[i]->geo) return STST_ERR_STATE;  // mapped-domain handles are solved one at a time
  }
  stst_batch_s *b = new (std::nothrow) stst_batch_s();
  if (!b) return STST_ERR_OOM;
  b->magic = STST_BATCH_MAGIC;
  b->count = count;
  b->hs.assign(handles, handles + count);
  // the branches run concurrently: no kernel of theirs may wait for CTAs that other branches keep off
  // the SMs, so the handles' mat-vecs stay one launch per level (no grid barriers)
  for (int i = 0; i < count; ++i) {
    handles[i]->no_fuse = 1;
    handles[i]->sys_plan.fuse = 0;
    handles[i]->lift_plan.fuse = 0;
  }
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {
    if (cudaStreamCreate(&b->stream) != cudaSuccess) {
      delete b;
      return STST_ERR_CUDA;
    }
    b->own_stream = 1;
  }
  int s = STST_OK;
  if (cudaMalloc(&b->params, sizeof(BatchParams)) != cudaSuccess ||
      cudaMalloc(&b->results, sizeof(BatchResult) * count) != cudaSuccess ||
      cudaMallocHost(&b->results_host, sizeof(BatchResult) * count) != cudaSuccess)
    s = STST_ERR_OOM;
  cudaGraph_t G = nullptr;
  if (s == STST_OK && cudaGraphCreate(&G, 0) != cudaSuccess) s = STST_ERR_CUDA;
  // tiles are chosen before capture (timing cannot run inside it); shapes seen before reuse the cache
  for (int i = 0; s == STST_OK && i < count; ++i) s = tune_modeprod(b->hs[i]);
  for (int i = 0; s == STST_OK && i < count; ++i) {
    // every problem's handle streams are idle: capturing on them records, it does not run
    if (cudaStreamSynchronize(b->hs[i]->stream) != cudaSuccess) s = STST_ERR_CUDA;
    if (s == STST_OK) s = add_branch(b, G, i, rhs[i], x[i]);
  }
  if (s == STST_OK) {
    cudaError_t e = cudaGraphInstantiate(&b->exec, G, 0);
    if (e != cudaSuccess) {
      stst_last_cuda = e;
      s = STST_ERR_CUDA;
    }
  }
  if (G) cudaGraphDestroy(G);
  if (s != STST_OK) {
    batch_free(b);
    return s;
  }
  *out = b;
  return STST_OK;
}

extern "C" int stst_batch_solve(stst_batch b, double tol, int maxit, int *iters, double *relres, int *status) {
  if (!b || b->magic != STST_BATCH_MAGIC) return STST_ERR_HANDLE;
  if (!(tol >= 0.0) || maxit < 1) return STST_ERR_ARG;
  BatchParams p;
  p.tol2 = tol * tol;
  p.maxit = maxit;
  p.pad = 0;
  STST_CUDA(cudaMemcpyAsync(b->params, &p, sizeof(p), cudaMemcpyHostToDevice, b->stream));
  STST_CUDA(cudaGraphLaunch(b->exec, b->stream));
  STST_CUDA(cudaMemcpyAsync(b->results_host, b->results, sizeof(BatchResult) * b->count, cudaMemcpyDeviceToHost,
                            b->stream));
  STST_CUDA(cudaStreamSynchronize(b->stream));
  int worst = STST_OK;
  for (int i = 0; i < b->count; ++i) {
    const BatchResult &r = b->results_host[i];
    if (iters) iters[i] = r.iters;
    if (relres) relres[i] = r.relres;
    if (status) status[i] = r.status;
    if (r.status != STST_OK && worst == STST_OK) worst = r.status;
    b->hs[i]->fd_ready = 1;
  }
  return worst;
}

extern "C" int stst_batch_destroy(stst_batch b) {
  if (!b || b->magic != STST_BATCH_MAGIC) return STST_ERR_HANDLE;
  batch_free(b);
  return STST_OK;
}
