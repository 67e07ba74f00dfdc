"""Training checkpoints resume exactly (host logic, CPU only).

The trainer's state is the context's FP32 parameters, AdamW moments and step
count, the next step index and the tile sampler's generator state. A stand-in
context with a deterministic step replaces the GPU here (the GPU run is checked
by tests/test_gpu_repair.py): a run interrupted after a checkpoint and resumed
in a fresh context must reproduce the uninterrupted run's remaining losses and
final weights bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_30741_gb300 import repair_train as T  # noqa: E402


class FakeCtx:
    """Context stand-in: AdamW on a deterministic gradient of the weights and the
    sampled tiles (float32 throughout, like the GPU's master weights)."""

    def __init__(self, fail_at=None):
        self.fail_at, self.calls = fail_at, 0

    def repair_load(self, w):
        self.w = np.asarray(w, np.float32).copy()
        self.m, self.v, self.k = np.zeros_like(self.w), np.zeros_like(self.w), 0

    def repair_state(self):
        return self.w.copy(), self.m.copy(), self.v.copy(), self.k

    def repair_load_state(self, w, m, v, k):
        self.w, self.m, self.v = (np.asarray(a, np.float32).copy() for a in (w, m, v))
        self.k = int(k)

    def repair_scratch(self, n):
        return None

    def repair_read(self, which=0):
        return self.w.copy()

    def repair_train_step(self, feat, target, plain, tiles, scratch=None, lr=1e-3, gate_weight=1.0, want_loss=True):
        if self.fail_at is not None and self.calls == self.fail_at:
            raise RuntimeError("interrupted")
        self.calls += 1
        t = tiles.numpy().astype(np.float64)
        phase = float(self.w[:16].astype(np.float64).sum()) + 1e-3 * float(t.sum())
        g = np.sin(phase + 1e-4 * np.arange(self.w.size)).astype(np.float32)
        self.k += 1
        b1, b2, eps = np.float32(0.9), np.float32(0.999), np.float32(1e-8)
        self.m = b1 * self.m + (1 - b1) * g
        self.v = b2 * self.v + (1 - b2) * g * g
        mh = self.m / np.float32(1 - 0.9 ** self.k)
        vh = self.v / np.float32(1 - 0.999 ** self.k)
        self.w = self.w - np.float32(lr) * mh / (np.sqrt(vh) + eps)
        loss = float(np.abs(self.w).mean())
        return [loss, loss, 0.0, 0.0]


class FakePairs:
    n = 3
    feat = target = plain = None

    def tile_tensor(self):
        return torch.arange(700, dtype=torch.int32)


def test_resume_reproduces_the_uninterrupted_run(tmp_path):
    pairs = FakePairs()
    w_full, h_full, _ = T.train(FakeCtx(), pairs, 30, 64, 1e-2, 5, log_every=1)
    ck = str(tmp_path / "ck_{step}.npz")
    with pytest.raises(RuntimeError):
        T.train(FakeCtx(fail_at=13), pairs, 30, 64, 1e-2, 5, log_every=1, checkpoint=ck, checkpoint_every=5)
    state = T.load_checkpoint(ck.format(step=10))
    assert state["next_step"] == 10 and state["adam_steps"] == 10
    w_res, h_res, _ = T.train(FakeCtx(), pairs, 30, 64, 1e-2, 5, log_every=1, resume=ck.format(step=10))
    assert [h[0] for h in h_res] == list(range(10, 30))
    assert h_res == h_full[10:]
    assert np.array_equal(w_res, w_full)


def test_resume_refuses_other_settings(tmp_path):
    ck = str(tmp_path / "ck.npz")
    T.train(FakeCtx(), FakePairs(), 6, 64, 1e-2, 5, log_every=1, checkpoint=ck, checkpoint_every=3)
    with pytest.raises(ValueError):
        T.train(FakeCtx(), FakePairs(), 6, 32, 1e-2, 5, log_every=1, resume=ck)  # another batch size
