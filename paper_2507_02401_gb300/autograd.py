"""torch.autograd wrappers of the linear operators of a plan.

Every operator here is linear, so each backward is the exact discrete
adjoint computed by the library's own kernels (paper Sec. 2.2 for K, Sec. 4
for E_s / E_s*):

    PatK    y = K x         backward  gx = K* gy
    PatKt   x = K* y        backward  gy = K gx
    PatEs   x = E_s u       backward  gu = E_s* gx
    PatEsT  u = E_s* x      backward  gx = E_s gu
    PatBatchK  [K_i x_i]    backward  [K_i* gy_i]   (one batched launch sequence)

Tensors are float32 on the plan's device; the calls run on the current CUDA
stream.  `reconstruction_loss` composes them into the regularised objective
J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 whose gradient is the residual
of the normal equations solved by `Plan.solve`.
"""
import torch

from . import _lib


def _stream():
    return torch.cuda.current_stream()


def _f32(t):
    return t.detach().to(dtype=torch.float32).contiguous()


class PatK(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, x):
        ctx.plan = plan
        y = torch.empty((plan.ns, plan.nt), device=x.device, dtype=torch.float32)
        _lib.pat_forward(plan.handle, _f32(x), y, _stream())
        return y

    @staticmethod
    def backward(ctx, gy):
        plan = ctx.plan
        gx = torch.empty(plan.shape, device=gy.device, dtype=torch.float32)
        _lib.pat_adjoint(plan.handle, _f32(gy), gx, _stream())
        return None, gx


class PatKt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, y):
        ctx.plan = plan
        x = torch.empty(plan.shape, device=y.device, dtype=torch.float32)
        _lib.pat_adjoint(plan.handle, _f32(y), x, _stream())
        return x

    @staticmethod
    def backward(ctx, gx):
        plan = ctx.plan
        gy = torch.empty((plan.ns, plan.nt), device=gx.device, dtype=torch.float32)
        _lib.pat_forward(plan.handle, _f32(gx), gy, _stream())
        return None, gy


class PatEs(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, s, u):
        ctx.plan, ctx.s = plan, float(s)
        x = torch.empty(plan.shape, device=u.device, dtype=torch.float32)
        _lib.pat_Es(plan.handle, ctx.s, _f32(u), x, _stream())
        return x

    @staticmethod
    def backward(ctx, gx):
        plan = ctx.plan
        gu = torch.empty(plan.N, device=gx.device, dtype=torch.float32)
        _lib.pat_EsT(plan.handle, ctx.s, _f32(gx), gu, _stream())
        return None, None, gu


class PatEsT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, s, x):
        ctx.plan, ctx.s = plan, float(s)
        u = torch.empty(plan.N, device=x.device, dtype=torch.float32)
        _lib.pat_EsT(plan.handle, ctx.s, _f32(x), u, _stream())
        return u

    @staticmethod
    def backward(ctx, gu):
        plan = ctx.plan
        gx = torch.empty(plan.shape, device=gu.device, dtype=torch.float32)
        _lib.pat_Es(plan.handle, ctx.s, _f32(gu), gx, _stream())
        return None, None, gx


class PatBatchK(torch.autograd.Function):
    """K of every instance of a Batch: forward runs the batched engine's K,
    backward its K* (inputs and outputs are B tensors each)."""

    @staticmethod
    def forward(ctx, batch, *xs):
        ctx.batch = batch
        ys = [torch.empty((p.ns, p.nt), device=x.device, dtype=torch.float32) for p, x in zip(batch.plans, xs)]
        _lib.pat_batch_forward(batch.handle, [_f32(x) for x in xs], ys, _stream())
        return tuple(ys)

    @staticmethod
    def backward(ctx, *gys):
        batch = ctx.batch
        gys = [torch.zeros((p.ns, p.nt), device="cuda") if g is None else g for p, g in zip(batch.plans, gys)]
        gxs = [torch.empty(p.shape, device=g.device, dtype=torch.float32) for p, g in zip(batch.plans, gys)]
        _lib.pat_batch_adjoint(batch.handle, [_f32(g) for g in gys], gxs, _stream())
        return (None,) + tuple(gxs)


def batch_K(batch, xs):
    return list(PatBatchK.apply(batch, *xs))


def K(plan, x):
    return PatK.apply(plan, x)


def Kt(plan, y):
    return PatKt.apply(plan, y)


def Es(plan, s, u):
    return PatEs.apply(plan, s, u)


def EsT(plan, s, x):
    return PatEsT.apply(plan, s, x)


class PatObjective(torch.autograd.Function):
    """J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 and its gradient
    E_s* K* (K E_s u - y) + alpha u, both computed by the library in one call
    (pat_objective); backward scales the stored gradient."""

    @staticmethod
    def forward(ctx, plan, u, y, alpha, s):
        grad = torch.empty(plan.N, device=u.device, dtype=torch.float32)
        J = _lib.pat_objective(plan.handle, _f32(y), alpha, s, _f32(u).reshape(-1), grad, _stream())
        ctx.save_for_backward(grad)
        ctx.u_shape = u.shape
        return torch.tensor(J, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        gu = (grad * gJ.to(torch.float32)).reshape(ctx.u_shape)
        return None, gu, None, None, None


def reconstruction_loss(plan, u, y, alpha, s):
    """J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 (float64 scalar, from the
    library); differentiable in u."""
    return PatObjective.apply(plan, u, y, alpha, s)
