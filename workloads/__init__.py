"""Seeded synthetic inputs shared by the decoder and its oracle.

Holds groups (Cayley tables), the seeded search for generating sets and local codes, and
per-qubit prior generators. Nothing here computes any part of the decoder itself.
"""
from .groups import Group, group, conjugacy_class_ids, generated_subgroup_size  # noqa: F401
from .search import (Instance, SplitMix64, candidate, paper_GA, paper_HA,  # noqa: F401
                     paper_instance, standard, STANDARD)
from .priors import errors_from_priors, per_qubit_priors  # noqa: F401
