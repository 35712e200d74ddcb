"""torch.autograd wrappers of the linear operators of a plan.

Every operator here is linear, so each backward is the exact discrete
adjoint computed by the library's own kernels (paper Sec. 2.2 for K, Sec. 4
for E_s / E_s*):

    PatK    y = K x         backward  gx = K* gy
    PatKt   x = K* y        backward  gy = K gx
    PatEs   x = E_s u       backward  gu = E_s* gx
    PatEsT  u = E_s* x      backward  gx = E_s gu

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


def K(plan, x):
    return PatK.apply(plan, x)


def Kt(plan, y):
    return PatKt.apply(plan, y)


def Es(plan, s, u):
    return PatEs.apply(plan, s, u)


def EsT(plan, s, x):
    return PatEsT.apply(plan, s, x)


def reconstruction_loss(plan, u, y, alpha, s):
    """J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 (accumulated in float64)."""
    r = K(plan, Es(plan, s, u)) - y
    return 0.5 * (r.double() ** 2).sum() + 0.5 * alpha * (u.double() ** 2).sum()
