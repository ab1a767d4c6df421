"""PyTorch's gradient of a real function of complex inputs is
dL/dRe + i dL/dIm (checked on |z|^2 and on a bilinear form), the same
convention as the factor gradients of eq. (25)-(27); CPU only."""
import numpy as np
import torch


def test_abs_squared():
    z = torch.tensor([1.5 - 0.5j, -2.0 + 3.0j], dtype=torch.complex128, requires_grad=True)
    (z.abs() ** 2).sum().backward()
    np.testing.assert_allclose(z.grad.numpy(), 2 * z.detach().numpy())


def test_real_part_of_bilinear_form_matches_wirtinger_convention():
    # L = Re(a^T z) for fixed complex a: dL/dRe z = Re a, dL/dIm z = -Im a -> grad = conj(a)
    a = torch.tensor([0.3 + 2.0j, -1.0 - 0.5j], dtype=torch.complex128)
    z = torch.zeros(2, dtype=torch.complex128, requires_grad=True)
    (a * z).sum().real.backward()
    np.testing.assert_allclose(z.grad.numpy(), np.conj(a.numpy()))
