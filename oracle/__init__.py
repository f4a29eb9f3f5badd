"""FP64 CPU oracle for the Flood complex filtration (test infrastructure).

This package is the independent checker of the CUDA path. It is plain, slow,
obviously correct numpy/scipy code that follows the paper's definitions:

  fps.py          farthest point sampling (§3.2, greedy k-centre), FP32 keys
  samples.py      barycentric grid P_sigma of Lemma 1 (§4.1)
  flood.py        f_P(sigma) = max_{p in P_sigma} min_{x in X} |p - x| (§4.1)
  random_flood.py the same for given point sets P_sigma (random draws, Lemma 4):
                  maximum over every face's set, faces enumerated explicitly
  grad.py         analytic subgradient of sum_sigma gamma_sigma f(sigma), central FD
  persistence.py  Z/2 boundary-matrix reduction (pairing), diagrams, bottleneck distance (§2)
  faces.py        faces and facet incidence of a set of tetrahedra, by definition

Only tests, the smoke check and the CPU-baseline leg of the benchmark may
import it. It shares no code with the CUDA path and imports nothing from the
product package; inputs (point clouds, simplex lists) are passed in as arrays.

Points may have d = 2..5 coordinates (fps.py and flood.py do not depend on d;
§5.3 varies it). Parity status: every function here is pinned by `-m "not gpu"`
tests against closed forms, invariants or brute force (tests/test_oracle_pins.py,
and tests/test_oracle_nd.py for d = 4, 5); none is "parity unpinned".
"""
from .fps import fps, fps_key
from .samples import compositions, interior_compositions, full_grid_count, interior_count, sample_points
from .flood import flood_values, nearest_distance, FloodResult
from .grad import analytic_gradient, finite_difference
from .random_flood import flood_values_random, analytic_gradient_random, total_random, RandomFloodResult
from .persistence import diagrams, bottleneck, bottleneck_within, persistence_pairs
from .faces import faces_by_definition, facet_rows

__all__ = [
    "fps", "fps_key", "compositions", "interior_compositions", "full_grid_count",
    "interior_count", "sample_points", "flood_values", "nearest_distance", "FloodResult",
    "analytic_gradient", "finite_difference", "diagrams", "bottleneck", "bottleneck_within",
    "persistence_pairs",
    "flood_values_random", "analytic_gradient_random", "total_random", "RandomFloodResult",
    "faces_by_definition", "facet_rows",
]
