"""The device complex reciprocal (the one every pivot of the factorisations uses) against
the exact reciprocal, through the C ABI (mhc_complex_reciprocal).

1/z = conj(z) / |z|^2: |z|^2 by one product and one fused multiply-add (relative error
<= 2u), 1/|z|^2 by two Newton-Raphson steps from the hardware approximation (<= 1u), and one
product per component (<= 1u): each component within 4u of the exact one to first order
(u = 2^-53); the test allows 5u.  Valid while |z|^2 stays a normal number:
2^-510 <= |z| <= 2^510.  The exact value comes from rational arithmetic (fractions).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def M():
    from paper_1411_3691_gb300 import build as B
    B.build()
    from paper_1411_3691_gb300 import mhc
    return mhc


def _cases():
    rng = np.random.default_rng(2024)
    mag = 2.0 ** rng.uniform(-500, 500, 1500)
    ang = rng.uniform(0, 2 * np.pi, 1500)
    z = mag * np.exp(1j * ang)
    # components of very different size: |im| / |re| from 1e-8 to 1e8
    ratio = 10.0 ** rng.uniform(-8, 8, 500)
    m2 = 2.0 ** rng.uniform(-400, 400, 500)
    z2 = m2 * (np.sign(rng.normal(size=500)) + 1j * ratio * np.sign(rng.normal(size=500)))
    special = np.array([1, -1, 1j, -1j, 3 + 4j, 2.0 ** 500, 2.0 ** -500, 1e-13 + 2e-13j,
                        complex(np.nextafter(1, 2), 0), 0.5 - 0.5j])
    return np.concatenate([z, z2, special]).astype(np.complex128)


def _exact(z):
    x, y = Fraction(float(z.real)), Fraction(float(z.imag))
    d = x * x + y * y
    return float(x / d), float(-y / d)


def test_complex_reciprocal_within_5u(M):
    z = _cases()
    got = M.mhc_complex_reciprocal(torch.from_numpy(z).cuda()).cpu().numpy()
    worst = 0.0
    for k in range(len(z)):
        er, ei = _exact(z[k])
        for g, e in ((got[k].real, er), (got[k].imag, ei)):
            if e == 0.0:
                assert g == 0.0, (z[k], g)
                continue
            rel = abs(g - e) / abs(e)
            worst = max(worst, rel / U)
            assert rel <= 5 * U, (z[k], g, e, rel / U)
    print(f"largest component error: {worst:.2f} u")
