"""Host-side logic of the serving loop (no GPU): byte accounting and the
seeded Poisson workload."""
import numpy as np

import bodex_inputs as I
from paper_2412_16490_gb300.serving import JobSpec, PoissonWorkload, job_bytes, object_bytes


def test_job_bytes_counts_the_resident_state():
    hand = I.hand_template("hand5")
    spec = JobSpec(hand, I.sphere_object(), np.zeros((100, hand.dof), np.float32), I.wrench_set(12))
    D, m, s = hand.dof, 5, 12
    assert job_bytes(spec) == 4 * (100 * (3 * D + s * 12 * m + s + 2) + s * 6)
    assert object_bytes(I.sphere_object()) == 0
    g = I.grid_object(1, n=16, h=0.008)
    assert object_bytes(g) == 4 * 16 ** 3


def test_poisson_workload_is_seeded_and_has_the_requested_rate():
    a = PoissonWorkload(n_jobs=40, rate=20.0, seed=5, grid_choices=(16, 24)).build()
    b = PoissonWorkload(n_jobs=40, rate=20.0, seed=5, grid_choices=(16, 24)).build()
    assert [s.arrival for s in a] == [s.arrival for s in b]
    assert all(np.array_equal(x.x0, y.x0) for x, y in zip(a, b))
    gaps = np.diff([0.0] + [s.arrival for s in a])
    assert 0.02 < gaps.mean() < 0.09  # mean 1/20 s
    assert {s.tag["template"] for s in a} <= {"hand3", "hand4x4", "hand5"}
    assert all(s.x0.shape[0] in (256, 512, 1024, 2048, 4096) for s in a)
