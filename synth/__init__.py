"""Seeded synthetic genome pairs for the seed-filter-extend hot path.

This package builds inputs only. It holds none of the method's arithmetic
(no seeding, no scoring, no extension): both the CPU oracle and the CUDA
library consume what it produces, and neither is imported here.
"""
from .rng import Stream, splitmix64
from .genome import (
    BASES, decode, encode_ascii, iid_bases, mutate, revcomp_codes, plant_repeats,
    plant_blocks, Pair,
)
from .workloads import (
    tiny_pair, plain_pair_10mb, batch_pairs, large_pair_100mb, WORKLOADS,
)

__all__ = [
    "Stream", "splitmix64", "BASES", "decode", "encode_ascii", "iid_bases", "mutate",
    "revcomp_codes", "plant_repeats", "plant_blocks", "Pair", "tiny_pair",
    "plain_pair_10mb", "batch_pairs", "large_pair_100mb", "WORKLOADS",
]
