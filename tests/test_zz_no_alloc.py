"""The allocation-free gradient entry point (hp_mlp_grad_noalloc) called
through the C ABI: two calls in a row match hp_mlp_grad, the existing entry
point, within the gradient tolerance of the other tests; oversize batches are
rejected.  Collected last so a run that stops at the first failure has run
everything else first."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_04644_gb300 import hp as _hp
    return _hp


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (B, 5)).astype(np.float32)
    t = rng.uniform(-1, 1, (B, 3)).astype(np.float32)
    return torch.tensor(x, device="cuda:0"), torch.tensor(t, device="cuda:0")


def test_noalloc_gradient_matches_existing_entry_point(hp):
    n_in, H, n_out = 5, 64, 3
    m = hp.hp_mlp_create(n_in, H, n_out, seed=21)
    try:
        n = hp.hp_mlp_info(m)[3]
        params = torch.tensor(hp.hp_mlp_params(m), device="cuda:0")
        # two calls in a row, the second smaller, so stale scratch from the first would show
        for B, seed in ((150, 1), (37, 2)):
            x, t = _batch(B, seed)
            g_ref = torch.empty(n, device="cuda:0")
            l_ref = torch.empty(1, device="cuda:0")
            hp.hp_mlp_grad(m, x, t, B, g_ref, l_ref)
            g = torch.full((n,), float("nan"), device="cuda:0")
            l = torch.full((1,), float("nan"), device="cuda:0")
            hp.hp_mlp_grad_noalloc(params, n_in, H, n_out, x, t, B, g, l)
            torch.cuda.synchronize()
            a, b = g.cpu().numpy(), g_ref.cpu().numpy()
            assert not np.isnan(a).any()
            assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max()
            assert abs(l.item() - l_ref.item()) <= 1e-5 * abs(l_ref.item())
    finally:
        hp.hp_mlp_destroy(m)


def test_noalloc_rejects_batches_beyond_its_scratch(hp):
    n_in, H, n_out = 5, 64, 3
    n = 5 * 64 + 64 + 64 * 64 + 64 + 3 * 64 + 3
    B = (1 << 20) // (n + 2 * H + n_out + 1) + 1
    params = torch.zeros(n, device="cuda:0")
    x, t = _batch(B, 3)
    g = torch.empty(n, device="cuda:0")
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mlp_grad_noalloc(params, n_in, H, n_out, x, t, B, g)
    assert ei.value.status == hp.HP_ERR_ARG
    assert "exceeds the fixed scratch" in hp.hp_last_error()
