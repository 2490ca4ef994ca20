"""Host logic of the autotuner: cache keys and candidate enumeration (no GPU)."""
import numpy as np

from paper_2205_11052_gb300.autotune import Autotuner, ensemble_key, workload_key


def test_workload_key_buckets_particles_per_cell():
    assert workload_key((32, 32, 32), 32 ** 3 * 60) == "32x32x32|ppc~64|B0|E0"
    assert workload_key((32, 32, 32), 32 ** 3 * 8, B=(0, 0, 5.0), wz2=1.0) == "32x32x32|ppc~8|B1|E1"


def test_ensemble_key_is_order_free():
    a = ((16, 16, 16), None, np.zeros((16 ** 3 * 8, 3)), None, -1.0)
    b = ((24, 24, 24), None, np.zeros((24 ** 3 * 32, 3)), None, -1.0)
    assert ensemble_key([a, b, a]) == ensemble_key([a, a, b])
    assert "x2" in ensemble_key([a, b, a])


def test_candidates_clip_the_tile_to_the_grid():
    t = Autotuner(space={"tile": [(8, 8, 8)], "sort_period": [2, 4]})
    c = list(t.candidates((16, 4, 1)))
    assert len(c) == 2 and all(x["tile"] == (8, 4, 1) for x in c)
