"""torch.autograd.Function around the adjoint-gradient entry point.

``Expectation`` holds an n-qubit state on the GPU, a parametrised circuit
(workloads.Gate records whose ``param`` fields index into a parameter vector)
and a Pauli-sum Hamiltonian. Its forward pass runs the circuit from |0...0>
and returns <H>; the backward pass calls qv_adjoint_grad, which runs the
circuit again and sweeps it in reverse (recomputation, no stored states).
"""
from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np
import torch

from . import qv
from .workloads import with_params


class Expectation:
    def __init__(self, n: int, gates: Sequence, terms: Sequence[Tuple[float, int, int]], nparams: int,
                 dtype: int = qv.QV_C64):
        self.n, self.gates, self.terms, self.nparams, self.dtype = n, list(gates), list(terms), nparams, dtype
        self.state = qv.StateVector(n, dtype)

    def _circuit(self, params: np.ndarray):
        return qv.gates_to_c(with_params(self.gates, params)), len(self.gates)

    def energy(self, params: np.ndarray) -> float:
        qv.qv_set_basis(self.state.h, 0)
        qv.qv_apply_circuit(self.state.h, self._circuit(params))
        return qv.qv_expect_pauli(self.state.h, self.terms)

    def grad(self, params: np.ndarray):
        """(d<H>/dparams, <H>) by the adjoint method."""
        qv.qv_set_basis(self.state.h, 0)
        return qv.qv_adjoint_grad(self.state.h, self._circuit(params), self.terms, self.nparams)

    def close(self):
        self.state.close()


class QvExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, model: Expectation):
        p = params.detach().to("cpu", torch.float64).numpy()
        ctx.model = model
        ctx.save_for_backward(params)
        return torch.tensor(model.energy(p), dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (params,) = ctx.saved_tensors
        g, _ = ctx.model.grad(params.detach().to("cpu", torch.float64).numpy())
        return torch.as_tensor(g, dtype=params.dtype, device=params.device) * grad_out, None


def expectation(params: torch.Tensor, model: Expectation) -> torch.Tensor:
    """<H>(params) as a differentiable torch scalar."""
    return QvExpectation.apply(params, model)
