"""Autotuner: searches the accumulator geometry on training matrices, stores
the choice per device, and the chosen options still give the oracle's result."""
import json

import pytest

from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu


def test_autotune_small_space(tmp_path, monkeypatch):
    from paper_2103_11991_gb300 import autotune as T
    monkeypatch.setattr(T, "training_problems",
                        lambda fam: [(A, A) for A in (I.stencil_3d(16, 16, 16, 27, 26.0, -1.0),)])
    space = {"team_vec_min_len": [8, 20], "use_window": [0, 1]}
    best, res = T.tune_family("stencil3d", space=space, reps=1)
    assert 2 <= len(res) <= 4 and set(best) == {"team_vec_min_len", "use_window"}
    assert res[json.dumps(best, sort_keys=True)] == min(res.values())
    assert all(v > 0 for v in res.values())
    path = tmp_path / "tuned.json"
    path.write_text(json.dumps({"stencil3d": {"options": best}}))
    assert T.tuned_options("stencil3d", path=str(path)) == best
    A = I.stencil_3d(12, 12, 12, 27, 26.0, -1.0)
    rp, ci, va, _, _ = run_gpu(A, A, **best)
    check_against_oracle(A, A, rp, ci, va, exact=True)


@pytest.mark.parametrize("sym_load,num_load", [(50, 25), (100, 50), (30, 10)])
def test_load_factor_options_keep_parity(sym_load, num_load):
    A = I.rmat(11, 16, seed=4)
    rp, ci, va, _, _ = run_gpu(A, A, sym_load_pct=sym_load, num_load_pct=num_load)
    check_against_oracle(A, A, rp, ci, va)
