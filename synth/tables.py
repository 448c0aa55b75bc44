"""Scoring data the method takes as input: the residue alphabet, BLOSUM62 and its
background amino-acid frequencies.

These are inputs (the substitution matrix is an argument of every call that scores
residues), not arithmetic of the method, so both the CPU oracle and the CUDA path are
handed the same table by the caller.

* Alphabet: the 24 symbols in the order of Sec. V-B (seed discovery), index 0..23.
  Sec. V-B's worked example RCQ -> 677 fixes this order.
* BLOSUM62: Henikoff & Henikoff, PNAS 89:10915 (1992) (the paper's citation for the
  matrix, Sec. IV-B and Sec. VI), in half-bit units, in its customary 24x24 layout
  (20 standard residues, then B, Z, X and the stop symbol *), which is the same order
  as the paper's alphabet.  The paper's own figure of the matrix (Fig. 6) did not
  survive; the entries it quotes in the text (A-A 4, C-C 9, A-S 1, A-C 0, A-G 0,
  Sec. IV-B) are checked by the tests.
* Background frequencies: the 20 single-residue frequencies underlying BLOSUM62 (same
  publication), rounded to three decimals; they sum to exactly 1.000.
"""
import numpy as np

ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"
N_SYMBOLS = 24
N_STANDARD = 20

_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0 -2 -1  0 -4
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3 -1  0 -1 -4
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3  3  0 -1 -4
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3  4  1 -1 -4
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1 -3 -3 -2 -4
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2  0  3 -1 -4
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3 -1 -2 -1 -4
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3  0  0 -1 -4
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3 -3 -3 -1 -4
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1 -4 -3 -1 -4
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2  0  1 -1 -4
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1 -3 -1 -1 -4
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1 -3 -3 -1 -4
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2 -2 -1 -2 -4
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2  0  0  0 -4
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0 -1 -1  0 -4
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3 -4 -3 -2 -4
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1 -3 -2 -1 -4
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4 -3 -2 -1 -4
-2 -1  3  4 -3  0  1 -1  0 -3 -4  0 -3 -3 -2  0 -1 -4 -3 -3  4  1 -1 -4
-1  0  0  1 -3  3  4 -2  0 -3 -3  1 -1 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -1 -1 -1 -2 -1 -1 -1 -1 -1 -1 -1 -1 -1 -2  0  0 -2 -1 -1 -1 -1 -1 -4
-4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4  1
"""

# A R N D C Q E G H I L K M F P S T W Y V
_BACKGROUND = (0.074, 0.052, 0.045, 0.054, 0.025, 0.034, 0.054, 0.074, 0.026, 0.068,
               0.099, 0.058, 0.025, 0.047, 0.039, 0.057, 0.051, 0.013, 0.032, 0.073)


def blosum62() -> np.ndarray:
    """24x24 int8 BLOSUM62 in ALPHABET order (a fresh copy on every call)."""
    rows = [list(map(int, ln.split())) for ln in _BLOSUM62_ROWS.strip().splitlines()]
    m = np.array(rows, dtype=np.int8)
    assert m.shape == (N_SYMBOLS, N_SYMBOLS)
    return m


def background() -> np.ndarray:
    """Background frequencies of the 20 standard residues (float64, ALPHABET order)."""
    return np.array(_BACKGROUND, dtype=np.float64)
