"""FP64 CPU oracle of the hierarchical merge-and-truncate SVD.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline legs of ``bench.py``; never by the product package.
"""
from .hmat import (ENERGY, FIXED_K, GAMMA, Refined, Result, Rule, Trace, block_svd,  # noqa: F401
                   grid, hmat_svd, iterative_improvement, mat_merge, mat_merge_orth, merge_tree,
                   normalise_signs, recover_left, relative_error, slab_step,
                   thin_svd, tree_schedule, truncated_svd)
from .metrics import (gap_prefix, leading_subspace_angle, orthonormality_defect,  # noqa: F401
                      principal_angle, sigma_rel_err, subspace_angles_grouped)
