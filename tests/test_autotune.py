"""The sweep autotuner: candidate generation, selection and its JSON cache (CPU, with a
fake solver and timer), and one real tuning run on the GPU."""
import numpy as np
import pytest

from paper_1208_3956_gb300 import autotune, helm, media


def test_candidates_surround_the_builtin_partition():
    Ny = 1055
    P0 = autotune.builtin_chunks(Ny)
    assert P0 == 96                      # the library's built-in count for this grid
    cands = autotune.candidates(Ny)
    Ps = sorted({P for P, _ in cands})
    assert P0 in Ps and min(Ps) < P0 < max(Ps)
    for P, G in cands:
        assert 1 <= G <= max(1, P // 2)
    assert autotune.candidates(79, dim=3) == [(0, 0)]
    # tiny grids: chunk counts clamped to (Ny+1)/2
    assert all(P <= 5 for P, _ in autotune.candidates(9))
    # wide panels: down to a sixth of the built-in count (one wave of 8 tiles needs P = 18)
    wide = sorted({P for P, _ in autotune.candidates(Ny, nrhs=32)})
    assert min(wide) == 16 and max(wide) == P0 and 24 in wide


class _Fake:
    closed = 0

    def __init__(self, P, G):
        self.P, self.G = P, G

    def close(self):
        _Fake.closed += 1


def test_tune_picks_the_fastest_skips_rejected_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    c = np.ones((20, 30))
    calls = []

    def make(P, G):
        if P == 7:
            raise helm.HelmError(-2, "out of memory")
        return _Fake(P, G)

    def measure(s, nrhs, reps):
        calls.append((s.P, s.G))
        return 10.0 + abs(s.P - 5) + 0.5 * abs(s.G - 2)

    cands = [(3, 1), (5, 1), (5, 2), (7, 2), (9, 3)]
    best = autotune.tune(c, 0.1, 2.0, 4, 3, 4, "mixed", cands=cands, make_solver=make, measure=measure,
                         path=path)
    assert (best["chunks"], best["sep_groups"]) == (5, 2)
    assert [t[:2] for t in best["tried"]] == [[3, 1], [5, 1], [5, 2], [9, 3]]
    assert _Fake.closed >= 4
    # second call: served from the cache, nothing measured
    calls.clear()
    again = autotune.tune(c, 0.1, 2.0, 4, 3, 4, "mixed", cands=cands, make_solver=make, measure=measure,
                          path=path)
    assert calls == [] and again["chunks"] == 5
    # another panel width is another key
    other = autotune.tune(c, 0.1, 2.0, 4, 3, 4, "mixed", nrhs=4, cands=cands[:2], make_solver=make,
                          measure=measure, path=path)
    assert other["chunks"] == 5 and calls


def test_tune_panel_minimises_time_per_rhs(tmp_path):
    class S:
        N, J, w_sub, precision = (50, 40), 4, 3, "mixed"

    def measure(s, B, reps):
        if B > 8:
            raise helm.HelmError(-2, "out of memory")
        return {1: 10.0, 2: 12.0, 4: 16.0, 8: 40.0}[B]

    r = autotune.tune_panel(S(), max_panel=32, path=str(tmp_path / "t.json"), measure=measure)
    assert r["panel"] == 4 and r["ms_per_rhs"] == pytest.approx(4.0)
    assert [t[0] for t in r["tried"]] == [1, 2, 4, 8]


@pytest.mark.gpu
def test_tune_on_the_device(tmp_path):
    n = (61, 45)
    c = media.smooth_medium(n, 3.0, 1.0, 2.0, 5)
    h = 1.0 / 32
    omega = media.omega_for(c, h, 8.0)
    best = autotune.tune(c, h, omega, 6, 5, 4, "mixed", reps=2, cands=[(3, 1), (5, 2)],
                         path=str(tmp_path / "t.json"))
    assert (best["chunks"], best["sep_groups"]) in [(3, 1), (5, 2)]
    assert len(best["tried"]) == 2 and all(t[2] > 0 for t in best["tried"])
    g = helm.HelmDD(c, h, omega, 6, 5, 4, "mixed", chunks=best["chunks"], sep_groups=best["sep_groups"]).factor()
    r = autotune.tune_panel(g, max_panel=4, reps=1, path=str(tmp_path / "t.json"))
    assert r["panel"] in (1, 2, 4)
    g.close()
