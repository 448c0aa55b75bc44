"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Holds the scoring tables the caller passes to the method and the planted-family
protein generators; none of the method's arithmetic lives here.
"""
from .tables import ALPHABET, N_STANDARD, N_SYMBOLS, background, blosum62
from .gen import (ProteinSet, families_1k, from_strings, planted_families,
                  random_proteins, zipf_100k, zipf_1m)
