"""Host logic of the differentiable diagrams (no GPU): the value bits of the
pair records decode to the field's values (float32 and float64, negative
and signed zeros included), and the persistence loss keeps exactly the
finite pairs above the threshold, with the gradient 2p at deaths and -2p at
births."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_13932_gb300 import autograd as ag  # noqa: E402


@pytest.mark.parametrize("dt,tdt,ubits", [(np.float32, torch.float32, np.uint32),
                                          (np.float64, torch.float64, np.uint64)])
def test_value_bits_decode_to_the_values(dt, tdt, ubits):
    vals = np.array([0.0, -0.0, 1.5, -2.25, 3e-38 if dt == np.float32 else 1e-300, -7.0,
                     np.inf, -np.inf], dtype=dt)
    bits = torch.from_numpy(vals.view(ubits).astype(np.uint64).view(np.int64))
    got = ag._bits_to_values(bits, tdt).numpy()
    assert np.array_equal(got.view(ubits), vals.view(ubits))


def test_persistence_loss_and_its_gradient():
    def diagram(birth, death, ess):
        b = torch.tensor(birth, dtype=torch.float64, requires_grad=True)
        d = torch.tensor(death, dtype=torch.float64, requires_grad=True)
        e = torch.tensor(ess, dtype=torch.bool)
        z = torch.zeros(len(birth), dtype=torch.int64)
        return ag.Diagram(b, d, e, z, z, z, z)
    d0 = diagram([0.0, 0.1, 0.2], [0.5, 0.105, 9.0], [False, False, True])
    d1 = diagram([0.0], [1.0], [False])
    d2 = diagram([0.3, 0.4], [0.9, 0.41], [False, False])
    loss = ag.persistence_loss([d0, d1, d2], threshold=0.01, dims=(0, 2))
    # kept: D0 (0.0, 0.5); D2 (0.3, 0.9); dropped: below the threshold, infinite, D1
    assert loss.item() == pytest.approx(0.5 ** 2 + 0.6 ** 2)
    loss.backward()
    assert d0.death.grad.tolist() == pytest.approx([1.0, 0.0, 0.0])
    assert d0.birth.grad.tolist() == pytest.approx([-1.0, 0.0, 0.0])
    assert d2.death.grad.tolist() == pytest.approx([1.2, 0.0])
    assert d2.birth.grad.tolist() == pytest.approx([-1.2, 0.0])
    assert d1.death.grad is None
