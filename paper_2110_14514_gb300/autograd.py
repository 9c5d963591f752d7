"""torch.autograd.Function whose forward is the GCP loss and whose backward is
the library's fused gradient kernel (arXiv 2110.14514 Sec. 2.2).

forward:  F = sum_i f(x_i, m_i) over a dense slice (exact), or the
          stratified-sample estimate of Alg. 5 over a sparse slice;
backward: dF/dA^(k) = Y_(k) Z_k diag(s) and dF/ds = Z' vec(Y) (eqs.
          gcp_grad_A, gcp_grad_lambda), scaled by grad_out on the device.

m is not stored between the passes: the backward launch recomputes the
Kruskal model values inside the fused kernel.  Only the gradient kernel runs;
no CPU fallback exists.
"""
import torch

from . import WANT_FACTORS, WANT_LOSS, WANT_TEMPORAL, SAMPLES_FACTOR_GRAD


class GCPLoss(torch.autograd.Function):
    """GCPLoss.apply(ctx, slice_kw, t, draw, s, *A) -> 0-dim float64 loss.

    ctx: a paper_2110_14514_gb300.Context (its loss, rank, dims and sampling
    parameters apply); slice_kw: dict(X=dense) or dict(idx=..., vals=...);
    t, draw: sample counter words (sparse slices).
    """

    @staticmethod
    def forward(fctx, gctx, slice_kw, t, draw, s, *A):
        _, _, f = gctx.gradient(s.detach(), [a.detach() for a in A], want=WANT_LOSS,
                                sample_set=SAMPLES_FACTOR_GRAD, t=t, draw=draw, **slice_kw)
        fctx.gctx = gctx
        fctx.slice_kw = slice_kw
        fctx.t, fctx.draw = t, draw
        fctx.save_for_backward(s, *A)
        return f.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        s, *A = fctx.saved_tensors
        scale = grad_out.detach().to(s.dtype).reshape(1).contiguous()
        G, gs, _ = fctx.gctx.gradient(s.detach(), [a.detach() for a in A], want=WANT_FACTORS | WANT_TEMPORAL,
                                      sample_set=SAMPLES_FACTOR_GRAD, t=fctx.t, draw=fctx.draw,
                                      y_scale=scale, **fctx.slice_kw)
        return (None, None, None, None, gs) + tuple(G)


def gcp_loss(gctx, s, A, X=None, idx=None, vals=None, t=1, draw=0):
    """Differentiable GCP loss of one slice at the point (s, A)."""
    kw = dict(X=X) if X is not None else dict(idx=idx, vals=vals)
    return GCPLoss.apply(gctx, kw, t, draw, s, *A)


class GraphedGCPLoss:
    """gcp_loss forward + backward captured once into a CUDA graph and replayed.

    The inputs are the static tensors given here (s, the factor matrices A, and the dense slice X
    or the sparse slice idx / vals): write new values into them and call replay().  After each
    replay the loss is in .loss and the gradients in s.grad and A[k].grad, which are also static.
    One replay runs the same two fused kernels as an eager forward + backward (the loss launch,
    then the gradient launch with the scale), without the host work of autograd and the binding.
    """

    def __init__(self, gctx, s, A, X=None, idx=None, vals=None, t=1, draw=0, warmup=2):
        import torch
        self.s, self.A = s, list(A)
        kw = dict(X=X) if X is not None else dict(idx=idx, vals=vals)

        def step():
            for v in self.A + [self.s]:
                v.grad = None
            loss = GCPLoss.apply(gctx, kw, t, draw, self.s, *self.A)
            loss.backward()
            return loss

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):   # the library's first launches (function attributes) happen here
            for _ in range(warmup):
                step()
        torch.cuda.current_stream().wait_stream(side)
        for v in self.A + [self.s]:
            v.grad = None
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss = GCPLoss.apply(gctx, kw, t, draw, self.s, *self.A)
            self.loss.backward()

    def replay(self):
        self.graph.replay()
        return self.loss
