"""Plain FP64 CPU oracle of the paper's retrieval and aggregation method.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct
statement of what the CUDA library computes, written from the paper (§3.1,
Algorithm 1; §3.2, Algorithm 2; §4) and from the readings listed with each
function. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the library never does, and this package
imports nothing from the library.

Modules:
  retrieval -- distance, exhaustive top-N, coarse-to-fine top-N, windows
  aggregate -- Algorithm 2 (2-D tile-density aggregation) and its centroid /
               softmax readings
  lowp      -- BF16 / FP8-e4m3 per-vector quantisation and the low-precision
               score + widened-shortlist re-rank heuristic
  soft      -- soft retrieval (softmax over negative weighted distances) with
               its analytic FP64 gradients
"""
from . import aggregate, lowp, retrieval, soft  # noqa: F401
