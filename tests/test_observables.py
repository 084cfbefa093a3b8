"""The package's S(k) and L(t) agree with the oracle's definitions."""
import numpy as np

from oracle import surrogate as OS
from paper_0902_3921_gb300 import inputs as I
from paper_0902_3921_gb300 import observables as OB


def test_observables_match_the_oracle():
    for seed in (0, 1):
        phi = np.tanh(5 * I.spinodal(2, 64, 64, seed=seed, amp=1.0))
        k1, S1 = OB.structure_factor(phi)
        k2, S2 = OS.structure_factor(phi)
        np.testing.assert_allclose(k1, k2, rtol=1e-14)
        np.testing.assert_allclose(S1, S2, rtol=1e-12, atol=1e-15)
        assert OB.domain_size(phi) == OS.domain_size(phi) or abs(
            OB.domain_size(phi) - OS.domain_size(phi)) < 1e-12
