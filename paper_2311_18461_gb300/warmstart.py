"""Learned warm start for families of solves (an extension: the paper's PCG starts from x0 = 0).

The network maps a problem's initial datum to a warm-start iterate. Its input is the datum's
coefficient vector c0 = M_s^{-1}(u0, B_j) (computed by `stst_rhs`), compressed to the coordinates of
an input basis; its output is the coordinates of x0 in an output basis of the solution space:
  x0 = Q_out^T sum_s S_s net_s(W_in^T Q_in c0),  S_s diagonal output scales, W_in the input whitening.
Stage s > 0 is trained on the remaining error of the stages before it, rescaled to unit RMS, so the
BF16 rounding of the weights (2^-9 relative) limits the cascade to about its product over the stages.
With a fixed potential the exact map c0 -> u is linear, so a linear network can learn it to the
accuracy of the two bases; PCG from x0 stays the arbiter of the result.

The pipeline orders library calls and owns device buffers; every numerical step runs in the library's
kernels; only the random draws (test matrices, minibatch permutations) and the learning-rate schedule are
host values:
  1. snapshots: `stst_rhs` gives (rhs, c0), the library's PCG solves; rows of Y and C0 hold them as reals;
  2. bases: `stst_pod_basis` on Y and on C0 (randomized subspace iteration, CholeskyQR2 with FP64 Gram);
  3. data: `stst_pod_project` gives features and targets; `stst_ws_whiten` whitens the features
     (Cholesky factor of their FP64 training covariance, folded into the rows of Q_in);
     `stst_ws_target_scale` scales every output coordinate to unit RMS (undone by each network's output
     scale) and weights each sample by 1 / ||coordinates||^2 (relative error);
  4. network: `stst_ws_train_step` over shuffled minibatches (Adam, cosine-decayed learning rate), each
     stage on the targets `stst_ws_cascade` forms from the error the stages before it left;
  5. inference: `stst_pod_project` -> `stst_ws_forward` per stage (accumulating) -> `stst_pod_expand` ->
     `stst_pcg_solve_guarded`,
     which restarts from x0 = 0 when the prediction is worse than zero.
"""
import math

import numpy as np

from . import _lib as B


class WarmStart:
    """Bases and network for one discretization (one `Problem`)."""

    def __init__(self, prob, K_in, K_out, hidden=(), stages=1, max_batch=256, seed=0):
        import torch
        self.torch = torch
        self.prob = prob
        self.N = prob.n_dof
        self.m = 2 * self.N
        self.m_in = 2 * prob.N_s
        self.K_in = int(K_in)
        self.K_out = int(K_out)
        self.sizes = [self.K_in] + [int(h) for h in hidden] + [self.K_out]
        self.max_batch = int(max_batch)
        self.nets = [B.stst_ws_create(self.sizes, self.max_batch, seed + 7919 * s, torch.cuda.current_stream())
                     for s in range(int(stages))]
        self.n_params = sum(B.stst_ws_num_params(w) for w in self.nets)
        self.history = []

    def close(self):
        for w in getattr(self, "nets", []):
            B.stst_ws_destroy(w)
        self.nets = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- 1. snapshots -------------------------------------------------------------------------------
    def collect(self, u0_list, tol=1e-8, maxit=200):
        """Right-hand side, c0 and PCG solution of every training datum (u0 on the quadrature grid)."""
        torch = self.torch
        n = len(u0_list)
        self.Y = torch.zeros((n, self.m), dtype=torch.float64, device="cuda")
        self.C0 = torch.zeros((n, self.m_in), dtype=torch.float64, device="cuda")
        Yc = self.Y.view(torch.complex128)
        Cc = self.C0.view(torch.complex128)
        rhs = self.prob.vec()
        its = []
        for i, u in enumerate(u0_list):
            u0 = u() if callable(u) else u
            B.stst_rhs(self.prob.h, None, u0, rhs, Cc[i])
            s, it, _ = B.stst_pcg_solve(self.prob.h, rhs, Yc[i], tol, maxit)
            if s != 0:
                raise RuntimeError(f"snapshot {i}: PCG status {s}")
            its.append(it)
        return its

    # ---- 2./3. bases, features, targets ---------------------------------------------------------------
    def fit(self, power_its=1, seed=0):
        """Both bases, the scaled features and targets, the per-sample weights."""
        torch = self.torch
        n = self.Y.shape[0]
        rng = np.random.default_rng(seed)
        Om = torch.as_tensor(rng.standard_normal((n, self.K_out), dtype=np.float32), device="cuda")
        self.Q_out = torch.empty((self.K_out, self.m), dtype=torch.float32, device="cuda")
        B.stst_pod_basis(self.Y, n, self.m, Om, self.K_out, power_its, self.Q_out)
        Om = torch.as_tensor(rng.standard_normal((n, self.K_in), dtype=np.float32), device="cuda")
        Q_in = torch.empty((self.K_in, self.m_in), dtype=torch.float32, device="cuda")
        B.stst_pod_basis(self.C0, n, self.m_in, Om, self.K_in, power_its, Q_in)
        T = torch.empty((n, self.K_out), dtype=torch.float32, device="cuda")
        F = torch.empty((n, self.K_in), dtype=torch.float32, device="cuda")
        B.stst_pod_project(self.Y, n, self.m, self.Q_out, self.K_out, T)
        B.stst_pod_project(self.C0, n, self.m_in, Q_in, self.K_in, F)
        # whitened features (Cholesky whitening, folded into the rows of Q_in), targets scaled to unit RMS
        # per coordinate, relative-error weights: all in the library
        self.F = torch.empty_like(F)
        B.stst_ws_whiten(F, n, self.K_in, self.F, Q_in, self.m_in)
        self.Q_in = Q_in
        self.T = torch.empty_like(T)
        self.so = torch.empty(self.K_out, dtype=torch.float64, device="cuda")
        self.W = torch.empty(n, dtype=torch.float32, device="cuda")
        B.stst_ws_target_scale(T, n, self.K_out, self.T, self.so, self.W)

    def _outputs(self, net, out):
        """The network's outputs on every training row (batches of max_batch) into out (n x K_out)."""
        n = self.F.shape[0]
        for i in range(0, n, self.max_batch):
            b = min(self.max_batch, n - i)
            B.stst_ws_forward(net, self.F[i:i + b], b, out[i:i + b])

    # ---- 4. training -------------------------------------------------------------------------------------
    def train(self, steps, batch=256, lr0=1e-3, lr1=1e-6, seed=0, log_every=0):
        """Each stage in turn: Adam over shuffled minibatches (a new permutation every epoch),
        cosine-decayed learning rate; stage s > 0 fits the rescaled error left by the stages before it
        (stst_ws_cascade keeps that error on the device)."""
        torch = self.torch
        n = self.T.shape[0]
        batch = min(batch, n, self.max_batch)
        rng = np.random.default_rng(seed)
        epochs = (steps * batch + n - 1) // n + 1
        K = self.K_out
        resid = torch.empty((n, K), dtype=torch.float64, device="cuda")
        targets = torch.empty((n, K), dtype=torch.float32, device="cuda")
        outs = torch.empty((n, K), dtype=torch.float32, device="cuda")
        scale = torch.empty(K, dtype=torch.float64, device="cuda")
        scale_prev = torch.empty(K, dtype=torch.float64, device="cuda")
        out_scale = torch.empty(K, dtype=torch.float32, device="cuda")
        for s, net in enumerate(self.nets):
            if s == 0:
                B.stst_ws_cascade(self.T, None, None, resid, n, K, scale, targets, self.so, out_scale)
            else:  # outs: what the previous stage predicts (its raw outputs, taken before its output scale)
                scale_prev, scale = scale, scale_prev
                B.stst_ws_cascade(None, outs, scale_prev, resid, n, K, scale, targets, self.so, out_scale)
            B.stst_ws_set_output_scale(net, None)
            perms = np.concatenate([rng.permutation(n)[: n - n % batch] for _ in range(epochs)]).astype(np.int32)
            perm = torch.as_tensor(perms, device="cuda")
            for k in range(steps):
                idx = perm[k * batch:(k + 1) * batch]
                lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * k / max(steps - 1, 1)))
                want = bool(log_every) and (k % log_every == 0 or k == steps - 1)
                loss = B.stst_ws_train_step(net, self.F, targets, self.W, idx, batch, lr, want_loss=want)
                if want:
                    self.history.append((s, k, loss))
            if s + 1 < len(self.nets):
                self._outputs(net, outs)
            # at inference the stage writes its share of the output-basis coordinates directly
            B.stst_ws_set_output_scale(net, out_scale)
        torch.cuda.synchronize()
        return self.history

    # ---- 5. inference ------------------------------------------------------------------------------------
    def predict(self, c0):
        """x0 (count x N complex128) for initial-datum coefficients c0 (count x N_s complex128)."""
        torch = self.torch
        c0 = c0.reshape(-1, self.m_in // 2)
        count = c0.shape[0]
        if count > self.max_batch:
            raise ValueError("more rows than max_batch")
        F = torch.empty((count, self.K_in), dtype=torch.float32, device="cuda")
        B.stst_pod_project(c0.contiguous().view(torch.float64), count, self.m_in, self.Q_in, self.K_in, F)
        C = torch.empty((count, self.K_out), dtype=torch.float32, device="cuda")
        for s, net in enumerate(self.nets):
            B.stst_ws_forward(net, F, count, C, 0.0 if s == 0 else 1.0)
        X = torch.empty((count, self.m), dtype=torch.float64, device="cuda")
        B.stst_pod_expand(self.Q_out, self.K_out, self.m, C, count, 1.0, 0.0, None, X)
        return X.view(torch.complex128)

    def solve(self, rhs, x0, tol=1e-8, maxit=200):
        """Guarded PCG from x0 (overwritten with the solution)."""
        s, it, rr, used = B.stst_pcg_solve_guarded(self.prob.h, rhs, x0, tol, maxit)
        return x0, s, it, rr, used
