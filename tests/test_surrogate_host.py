"""Host-side logic of the surrogate driver (no GPU): the symmetry
augmentation of the training fields must commute with the conduction
operator (checked with the FP64 oracle), i.e. transform (T, b) the way the
physics transforms under the cube's symmetries."""
import numpy as np
import pytest

from oracle import Problem


def test_augmentation_commutes_with_the_operator(orc):
    torch = pytest.importorskip("torch")
    from paper_1702_05487_gb300.surrogate import augment
    import workloads
    n = 12
    T, b = workloads.tangled_box(n, n, n, 42)
    P = Problem((n, n, n), kappa_model="spitzer", kappa_par0=0.02, kappa_perp_ratio=0.05)
    M = orc.apply_M(P, T, b)
    for seed in range(6):
        Tt, bt = augment(torch.from_numpy(T), torch.from_numpy(b), np.random.default_rng(seed))
        Mt, _ = augment(torch.from_numpy(M), torch.from_numpy(b), np.random.default_rng(seed))
        got = orc.apply_M(P, Tt.numpy(), bt.numpy())
        assert np.max(np.abs(got - Mt.numpy())) < 1e-12 * np.max(np.abs(M)), seed
