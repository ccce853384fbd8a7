"""Host logic of the autotuner on CPU: the coordinate descent over the option
space finds the minimum of a separable cost, never times a candidate that
breaks the threshold order (team below CTA), and starts from the defaults."""
import json

from paper_2103_11991_gb300 import autotune as T


def _fake(monkeypatch, cost):
    calls = []
    monkeypatch.setattr(T, "training_problems", lambda fam: [(None, None)])

    class _D:
        @staticmethod
        def from_host(M):
            return M

    monkeypatch.setattr(T.K, "DeviceCSR", _D)

    def timed(a, b, opts, reps=3):
        calls.append(dict(opts))
        return cost(opts)

    monkeypatch.setattr(T, "_time_plain", timed)
    return calls


def test_descent_finds_separable_minimum(monkeypatch):
    target = {"team_vec_min_len": 20, "sym_load_pct": 50, "num_load_pct": 25, "use_window": 0,
              "sym_team_max_flop": 6144, "sym_cta_max_flop": 12288, "num_team_max_nnz": 512,
              "num_cta_max_nnz": 8192}

    def cost(o):
        return 1.0 + sum(abs(T.SPACE[k].index(o[k]) - T.SPACE[k].index(target[k])) for k in T.SPACE)

    calls = _fake(monkeypatch, cost)
    best, res = T.tune_family("stencil3d")
    assert best == target
    assert calls[0] == T.DEFAULTS
    assert all(T._valid(c) for c in calls)
    assert res[json.dumps(best, sort_keys=True)] == 1.0
    # far fewer timings than the whole product of the axes
    assert len(res) < 60


def test_descent_respects_threshold_order(monkeypatch):
    # the cheapest point would put the team threshold above the CTA one
    def cost(o):
        return -o["num_team_max_nnz"] + 0.5 * o["num_cta_max_nnz"]

    calls = _fake(monkeypatch, cost)
    best, _ = T.tune_family("stencil3d")
    assert all(c["num_team_max_nnz"] < c["num_cta_max_nnz"] for c in calls)
    valid = [cost(dict(best, num_team_max_nnz=a, num_cta_max_nnz=b))
             for a in T.SPACE["num_team_max_nnz"] for b in T.SPACE["num_cta_max_nnz"] if a < b]
    assert best["num_team_max_nnz"] < best["num_cta_max_nnz"] and cost(best) == min(valid)
