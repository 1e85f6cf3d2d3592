"""Host logic of the binding's autograd wrapper of mlmd_propagate_adjoint,
with the ABI call replaced by a fake that returns known gradients (no GPU)."""
import numpy as np
import torch

from paper_2509_00966_gb300 import mlmd


class _FakeDomain:
    n_grid = 5
    handle = None

    def __init__(self):
        self.V = None

    def set_potential(self, v):
        self.V = np.array(v)


def test_excitation_loss_backward_chains_both_gradients(monkeypatch):
    dA_known = np.arange(12, dtype=np.float64).reshape(4, 3) * 0.1
    dV_known = np.linspace(-1.0, 1.0, 5)
    seen = {}

    def fake_adjoint(h, A, ckpt_every, n_grid, dL_dV):
        seen["A"], seen["ckpt"] = np.array(A), ckpt_every
        dL_dV.copy_(torch.from_numpy(dV_known))
        return 7.5, dA_known.copy(), dL_dV

    monkeypatch.setattr(mlmd, "propagate_adjoint", fake_adjoint)
    dom = _FakeDomain()
    A0 = torch.ones(4, 3, dtype=torch.float64)
    s = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    V = torch.full((5,), 0.25, dtype=torch.float64, requires_grad=True)
    loss = mlmd.excitation_loss(dom, s * A0, V, ckpt_every=3)
    assert loss.item() == 7.5 and loss.dtype == torch.float64
    np.testing.assert_array_equal(seen["A"], 2.0 * np.ones((4, 3)))
    assert seen["ckpt"] == 3
    np.testing.assert_array_equal(dom.V, np.full(5, 0.25))     # V became the domain's potential
    (3.0 * loss).backward()
    np.testing.assert_allclose(V.grad.numpy(), 3.0 * dV_known)
    assert abs(s.grad.item() - 3.0 * float(np.sum(dA_known))) < 1e-12
