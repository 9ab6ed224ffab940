"""The library's training loop (cm_net_train) and checkpoints (cm_net_save /
cm_net_load): the loop equals its steps taken one by one, and a run split by
a checkpoint equals the run in one piece, bit for bit."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2204_07921_gb300 as cm  # noqa: E402
from paper_2204_07921_gb300 import warmstart as ws  # noqa: E402

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix(z):
    """SplitMix64's output function (Steele, Lea and Flood, 2014)."""
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def batch_of(seed, t, n, batch):
    state = mix(seed + GAMMA * (t + 1))
    perm = list(range(n))
    out = []
    for j in range(batch):
        r = j + mix(state + GAMMA * (j + 1)) % (n - j)
        perm[j], perm[r] = perm[r], perm[j]
        out.append(perm[j])
    return out


def pairs(n=7, side=24, seed=3):
    rng = np.random.default_rng(seed)
    F = rng.random((n, side, side), dtype=np.float32)
    U = (F * 0.8 + 0.1).astype(np.float32)
    return torch.from_numpy(F).cuda(), torch.from_numpy(U).cuda()


def fresh(seed=1):
    return ws.Net(ws.init_params(seed, zero_last=False))


def test_loop_equals_single_steps():
    F, U = pairs()
    a, b = fresh(), fresh()
    steps, batch, lr, lrf, seed = 5, 3, 2e-3, 1e-4, 11
    log = a.train_native(F, U, steps, batch, lr, lrf, seed=seed, log_every=1)
    T = steps
    lr32, lrf32 = float(np.float32(lr)), float(np.float32(lrf))
    losses = []
    for t in range(steps):
        idx = batch_of(seed, t, F.shape[0], batch)
        it = torch.tensor(idx, device="cuda")
        a_t = lrf32 + 0.5 * (lr32 - lrf32) * (1.0 + np.cos(np.pi * t / max(1, T - 1)))
        losses.append(b.train_step(F.index_select(0, it).contiguous(),
                                   U.index_select(0, it).contiguous(), float(np.float32(a_t))))
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    assert log["steps"] == list(range(steps))
    np.testing.assert_array_equal(log["losses"], losses)
    assert log["loss_first"] == losses[0] and log["loss_last"] == losses[-1]


def test_checkpoint_resume_is_exact(tmp_path):
    F, U = pairs(9, 20, 5)
    whole = fresh(2)
    whole.train_native(F, U, 6, 4, 3e-3, 2e-4, seed=5, total_steps=6)
    first = fresh(2)
    first.train_native(F, U, 3, 4, 3e-3, 2e-4, seed=5, total_steps=6)
    path = os.path.join(tmp_path, "net.ckpt")
    first.save_checkpoint(path)
    resumed = fresh(7)                  # other parameters: the checkpoint replaces them
    resumed.load_checkpoint(path)
    assert np.array_equal(resumed.get_params(), first.get_params())
    resumed.train_native(F, U, 3, 4, 3e-3, 2e-4, seed=5, total_steps=6, start_step=3)
    torch.cuda.synchronize()
    assert np.array_equal(resumed.get_params(), whole.get_params())


def test_checkpoint_rejects_damaged_files(tmp_path):
    net = fresh(4)
    path = os.path.join(tmp_path, "net.ckpt")
    net.save_checkpoint(path)
    raw = bytearray(open(path, "rb").read())
    assert raw[:8] == b"CMNETCK1" and len(raw) == 24 + 3 * 4 * ws.N_PARAMS + 4
    before = net.get_params()
    cases = {"flip": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], "short": raw[:-8],
             "magic": b"XMNETCK1" + raw[8:]}
    for name, data in cases.items():
        bad = os.path.join(tmp_path, name)
        open(bad, "wb").write(bytes(data))
        with pytest.raises(cm.CMError) as e:
            net.load_checkpoint(bad)
        assert e.value.code == cm.CM_ERR_INVALID, name
    with pytest.raises(cm.CMError):
        net.load_checkpoint(os.path.join(tmp_path, "missing"))
    assert np.array_equal(net.get_params(), before)
