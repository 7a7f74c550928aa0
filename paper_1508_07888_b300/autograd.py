"""Differentiable ionisation history: torch.autograd.Function over
rt_step (forward) and rt_adjoint (backward).

    run = HistoryRun(params, box_state, initial_state, nsteps, ckpt_every)
    X = ionisation_history(Q, n0, run)          # X[t] after step t+1
    loss = ((X - X_target) ** 2).mean()
    loss.backward()                             # Q.grad, n0.grad

Q: float64 tensor of the source luminosities (photons/s, the order of
run.cells); n0: float64 CUDA tensor [nz, ny, nx] of the density (cm^-3).
The forward pass restarts from the stored initial state every call.  The
gradient comes from the library's hand-written adjoint (FP64, periodic box,
branch decisions of the forward pass frozen).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class HistoryRun:
    """A single-box FP64 handle, its initial state and the run length."""

    def __init__(self, params: B.rt_params, state: B.BoxState, cells, nsteps: int,
                 ckpt_every: int = 20):
        assert params.precision in (B.RT_PREC_FP64, B.RT_PREC_FP64_STRICT)
        self.state = state
        self.U0 = state.U.clone()
        self.x0 = state.xHI.clone()
        self.T0 = state.T.clone()
        self.cells = np.ascontiguousarray(cells, dtype=np.int64)
        self.nsteps = int(nsteps)
        self.ckpt = int(ckpt_every)
        self.solver = B.Solver(params, [state])

    def forward(self, Q: torch.Tensor, n0: torch.Tensor) -> torch.Tensor:
        st = self.state
        st.n0.copy_(n0.detach().to(device=st.n0.device, dtype=st.n0.dtype))
        self.solver.set_sources(0, self.cells, Q.detach().cpu().double().numpy())
        st.U.copy_(self.U0)
        st.xHI.copy_(self.x0)
        st.T.copy_(self.T0)
        hist = torch.zeros((self.nsteps, 1, B.RT_NDIAG), dtype=torch.float64, device=st.U.device)
        code = self.solver.step(self.nsteps, hist)
        if code != B.RT_OK:
            raise B.RTError(code, B.rt_last_error(self.solver.h))
        return hist[:, 0, 0].clone()

    def backward(self, gX: torch.Tensor):
        st = self.state
        g = gX.detach().to(device=st.U.device, dtype=torch.float64).contiguous()
        dn0 = torch.zeros_like(st.xHI)
        code, dQ = B.rt_adjoint(self.solver.h, self.U0.data_ptr(), self.x0.data_ptr(),
                                self.T0.data_ptr(), self.nsteps, self.ckpt, g.data_ptr(),
                                len(self.cells), dn0.data_ptr())
        if code != B.RT_OK:
            raise B.RTError(code, B.rt_last_error(self.solver.h))
        return torch.from_numpy(dQ.copy()), dn0

    def close(self):
        self.solver.close()


class IonisationHistory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, n0, run: HistoryRun):
        ctx.run = run
        ctx.q_device, ctx.q_dtype = Q.device, Q.dtype
        return run.forward(Q, n0)

    @staticmethod
    def backward(ctx, gX):
        dQ, dn0 = ctx.run.backward(gX)
        return dQ.to(device=ctx.q_device, dtype=ctx.q_dtype), dn0, None


def ionisation_history(Q: torch.Tensor, n0: torch.Tensor, run: HistoryRun) -> torch.Tensor:
    return IonisationHistory.apply(Q, n0, run)
