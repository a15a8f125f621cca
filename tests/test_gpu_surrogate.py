"""Surrogate MLP kernels (tcgen05 BF16, FP32 accumulation) against the FP64
reference network of oracle/mlp.py.

The weights are BF16-representable, so both sides use the same network; the
GPU rounds the normalised input and every hidden activation to BF16 (relative
2^-9 per element), which bounds the stated agreement: 1e-2 relative L2 on the
outputs and on the loss, 3e-2 relative L2 per gradient tensor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build   # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sur():
    build.build()
    from paper_2106_08040_gb300 import surrogate
    return surrogate


def random_net(sur, seed):
    s = sur.Surrogate(seed=seed)
    rng = np.random.default_rng(seed + 1)
    for l in range(sur.LAYERS):
        w = s.Wm[l].cpu().numpy()
        s.Wm[l].copy_(torch.from_numpy(w).to(torch.bfloat16).float())
        s.bm[l].copy_(torch.from_numpy(rng.normal(0, 0.1, size=sur.NL[l]).astype(np.float32)))
    s.in_shift.copy_(torch.from_numpy(rng.normal(0, 0.5, size=7).astype(np.float32)))
    s.in_scale.copy_(torch.from_numpy(rng.uniform(0.5, 2.0, size=7).astype(np.float32)))
    s.out_shift.copy_(torch.from_numpy(rng.normal(0, 1.0, size=800).astype(np.float32)))
    s.out_scale.copy_(torch.from_numpy(rng.uniform(0.5, 2.0, size=800).astype(np.float32)))
    s.refresh()
    torch.cuda.synchronize()
    return s


def oracle_params(s):
    st = s.state()
    return {"W": [w.astype(np.float64) for w in st["Wm"]], "b": [b.astype(np.float64) for b in st["bm"]],
            "in_shift": st["in_shift"].astype(np.float64), "in_scale": st["in_scale"].astype(np.float64),
            "out_shift": st["out_shift"].astype(np.float64), "out_scale": st["out_scale"].astype(np.float64)}


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("q", [1, 129, 300])
def test_infer_matches_oracle(sur, q):
    from oracle import mlp
    s = random_net(sur, 3)
    x = np.random.default_rng(q).normal(size=(q, 7))
    y = s.infer(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    torch.cuda.synchronize()
    assert s.error_flag() == 0
    y_or, _ = mlp.forward(oracle_params(s), x.astype(np.float32).astype(np.float64))
    assert rel(y, y_or) < 1e-2, rel(y, y_or)
    per_query = np.linalg.norm(y - y_or, axis=1) / np.linalg.norm(y_or, axis=1)
    assert per_query.max() < 3e-2


@pytest.mark.parametrize("q", [136, 256])
def test_grad_matches_oracle(sur, q):
    from oracle import mlp
    s = random_net(sur, 4)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(q, 7)).astype(np.float32)
    y = rng.normal(size=(q, 800)).astype(np.float32)
    loss = float(s.grad(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).item())
    torch.cuda.synchronize()
    assert s.error_flag() == 0
    l_or, gW, gb = mlp.loss_and_grad(oracle_params(s), x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - l_or) / l_or < 1e-2, (loss, l_or)
    for l in range(sur.LAYERS):
        assert rel(s.gW[l].cpu().numpy(), gW[l]) < 3e-2, (l, rel(s.gW[l].cpu().numpy(), gW[l]))
        assert rel(s.gb[l].cpu().numpy(), gb[l]) < 3e-2, (l, rel(s.gb[l].cpu().numpy(), gb[l]))


def test_training_fits_a_teacher_network(sur):
    teacher = random_net(sur, 11)
    rng = np.random.default_rng(12)
    x = torch.from_numpy(rng.normal(size=(8192, 7)).astype(np.float32)).cuda()
    y = teacher.infer(x).clone()
    student = sur.Surrogate(seed=13)
    student.in_shift.copy_(teacher.in_shift)
    student.in_scale.copy_(teacher.in_scale)
    student.out_shift.copy_(teacher.out_shift)
    student.out_scale.copy_(teacher.out_scale)
    hist = student.fit(x, y, steps=300, batch=1024, lr=1e-3, log_every=50)
    torch.cuda.synchronize()
    assert student.error_flag() == 0
    assert hist[-1][1] < 0.1 * hist[0][1], hist
