"""Host logic of the learned screen's calibration (no GPU): with an engine
whose K error grows with each threshold, calibrate() keeps the largest skip
threshold within its budget, then the largest tier threshold keeping both
within theirs, stops at the first threshold over budget and stores both."""
import json
import types

import numpy as np

import paper_2303_14280_gb300.train_screen as ts


class _FakeEngine:
    calls = []

    def __init__(self, basis, grid, screen="link", learned_skip=-99.0, learned_fp32=-99.0, **form):
        self.learned = screen == "learned"
        self.skip, self.fp32 = learned_skip, learned_fp32
        _FakeEngine.calls.append((self.learned, self.skip, self.fp32))

    def screen_load(self, w):
        pass

    def set_density(self, P):
        pass

    def build_K(self):
        err = 0.0
        if self.learned:
            err += 10.0 ** (self.skip + 1.6)               # skip: -10.5 -> 1.26e-9, -10.25 -> 2.2e-9
            if self.fp32 > -50:
                err += 10.0 ** (self.fp32 - 4.8)           # tier: -4.0 -> 1.6e-9, -3.75 -> 2.8e-9
        return np.full((3, 3), 0.5 + err)

    def stats(self):
        return {"pairs_learned_skipped": 1, "pairs_kept_fp32": 2, "pairs_kept": 3}

    def close(self):
        pass


def test_calibration_picks_the_largest_thresholds_within_budget(tmp_path, monkeypatch):
    fake = types.SimpleNamespace(Engine=_FakeEngine)
    monkeypatch.setattr(ts, "instance", lambda seed, dev: types.SimpleNamespace(basis=None, grid=None, P=None))
    _FakeEngine.calls = []
    out = tmp_path / "w.npz"
    args = types.SimpleNamespace(instances=20, out=str(out))
    ts.calibrate(fake, np.zeros(16, dtype=np.float32), {"blocks": 0}, args, None)
    with np.load(out) as z:
        thr = float(z["threshold"])
        meta = json.loads(str(z["meta"]))
    assert thr == -10.5                                    # 1.26e-9 <= 2e-9 < 2.2e-9
    assert meta["fp32_threshold"] == -4.0                  # 1.26e-9 + 1.6e-9 <= 3e-9 < 1.26e-9 + 2.8e-9
    assert meta["holdout_seed"] == ts.TRAIN_SEED0 + 20
    skips = [c[1] for c in _FakeEngine.calls if c[0] and c[2] == -99.0]
    assert skips == [-12.0, -11.5, -11.0, -10.75, -10.5, -10.25]   # stops at the first over budget
    tiers = [c[2] for c in _FakeEngine.calls if c[0] and c[2] != -99.0]
    assert tiers[-1] == -3.75 and all(c[1] == -10.5 for c in _FakeEngine.calls if c[0] and c[2] != -99.0)
    assert len(meta["calibration"]) == 6 and len(meta["calibration_fp32"]) == len(tiers)
