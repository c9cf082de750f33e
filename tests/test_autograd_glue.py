"""The torch.autograd layer's marshalling, on the CPU with a stand-in for the library-backed
Problem: forward hands b and the entry values to the problem and returns its iterate; backward
hands the output gradients to mcsdp_backward's binding and routes its results to b and the
entry values (and nothing else).  The arithmetic itself is tested on the GPU."""
import numpy as np
import torch

import paper_1310_6919_gb300.autograd as ag


class FakeProblem:
    made = []

    def __init__(self, n, m, b, mat, row, col, val, **options):
        self.args = (n, m, np.array(b), np.array(mat), np.array(row), np.array(col),
                     np.array(val), options)
        self.z0 = None
        FakeProblem.made.append(self)

    def set_iterate(self, X, z):
        self.z0 = z

    def solve(self):
        self.solved = True
        return {"status": 0}

    def get_iterate(self):
        return (torch.arange(5, dtype=torch.float64), torch.tensor([1.0, 2.0], dtype=torch.float64),
                None)

    def backward(self, gX, gz):
        self.grads = (gX.clone(), gz.clone())
        return {"gb": torch.tensor([10.0, 20.0], dtype=torch.float64),
                "g_entries": torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64)}


def test_forward_and_backward_marshalling(monkeypatch):
    monkeypatch.setattr(ag, "Problem", FakeProblem)
    FakeProblem.made.clear()
    b = torch.tensor([1.0, 1.0], dtype=torch.float64, requires_grad=True)
    val = torch.tensor([0.5, -0.25, 1.0], dtype=torch.float64, requires_grad=True)
    mat, row, col = [0, 1, 2], [0, 0, 1], [0, 1, 1]
    X, z = ag.solve_layer(b, val, 2, 2, mat, row, col, z0=torch.zeros(2), device=-1, relax=0)
    P = FakeProblem.made[-1]
    assert P.solved and P.z0 is not None
    n, m, bb, mm, rr, cc, vv, opts = P.args
    assert (n, m) == (2, 2) and np.array_equal(bb, [1.0, 1.0]) and np.array_equal(vv, [0.5, -0.25, 1.0])
    assert opts == {"device": -1, "relax": 0}
    assert torch.equal(X, torch.arange(5, dtype=torch.float64))
    loss = (X * torch.arange(5, dtype=torch.float64)).sum() + 3.0 * z.sum()
    loss.backward()
    gX, gz = P.grads
    assert torch.equal(gX, torch.arange(5, dtype=torch.float64))
    assert torch.equal(gz, torch.tensor([3.0, 3.0], dtype=torch.float64))
    assert torch.equal(b.grad, torch.tensor([10.0, 20.0], dtype=torch.float64))
    assert torch.equal(val.grad, torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64))
