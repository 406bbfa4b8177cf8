"""Host logic of the Gym-style environment (no GPU): the task ids are the header's, and the
reference path of every env starts within the spawn radius of the origin (checked with the
oracle's own task reference), at phases spread over the circle."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_14117_gb300.env import TASKS, task_centres

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_task_ids_are_the_headers():
    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    ids = {m.group(1).lower(): int(m.group(2))
           for m in re.finditer(r"#define MG_TASK_(\w+) (\d+)", text)}
    assert ids == TASKS


@pytest.mark.parametrize("task", sorted(TASKS))
@pytest.mark.parametrize("spawn", [0.0, 0.5])
def test_reference_starts_near_the_origin(task, spawn):
    n, radius = 2000, 2.0
    c = task_centres(task, n, radius, seed=7, spawn_radius=spawn)
    start = np.stack([O.task_reference(TASKS[task], c[e], radius, 0.3, 0.1, 0.0)
                      for e in range(n)])
    d = np.linalg.norm(start, axis=1)
    assert d.max() <= spawn + 1e-12
    if spawn > 0:
        # uniform in the ball: the median distance is spawn / 2^(1/3)
        assert abs(np.median(d) - spawn * 0.5 ** (1 / 3)) < 0.03 * spawn
    phase = c[:, 3]
    assert phase.min() >= 0.0 and phase.max() < 2 * np.pi
    counts, _ = np.histogram(phase, bins=8, range=(0, 2 * np.pi))
    assert counts.min() > 0.8 * n / 8


def test_unknown_task_rejected():
    with pytest.raises(ValueError):
        task_centres("orbit", 4, 2.0, 0)
