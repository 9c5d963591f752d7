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
