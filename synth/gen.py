"""Seeded synthetic protein sets with planted families.

This module only draws inputs; it holds none of the method's arithmetic (no k-mers,
no candidate discovery, no alignment, no filtering).  Both the CPU oracle and the
CUDA path read what it returns.

The paper measures on Metaclust50 subsets and on SCOPe (Sec. VI), which are not
available here; these generators stand in for them with the shapes the workloads
call for:

* root lengths log-normal with median 300 (mu = ln 300) and sigma = 0.6, clipped to
  the workload's length range;
* residues i.i.d. from the BLOSUM62 background over the 20 standard amino acids;
* a family member copies its root, substitutes 30% of positions (replacement b != a
  drawn with probability proportional to p_b * 2^(s(a,b)/2), BLOSUM62 being in
  half-bit units), then applies insertion/deletion events at a rate of 0.05/3 per
  position (half insertions, half deletions, geometric lengths of mean 3), so about
  5% of residues are touched; inserted residues come from the background;
* members are re-clipped to the length range (truncated, or padded with background
  residues); roots themselves are not emitted; singletons are fresh roots;
* the whole set is shuffled, and every sequence carries its family id.

Sequences are returned as ASCII letters of the 24-symbol alphabet (only the 20
standard letters occur), concatenated, with int64 offsets.
"""
from dataclasses import dataclass, field

import numpy as np

from .tables import ALPHABET, N_STANDARD, background, blosum62

_LETTERS = np.frombuffer(ALPHABET.encode("ascii"), dtype=np.uint8)


@dataclass
class ProteinSet:
    ascii: np.ndarray      # uint8 [R] concatenated residues (ASCII letters)
    offsets: np.ndarray    # int64 [n+1]
    family: np.ndarray     # int32 [n] planted family id (singletons: unique ids)
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def seq(self, i: int) -> str:
        return self.ascii[self.offsets[i]:self.offsets[i + 1]].tobytes().decode("ascii")

    def subset(self, ids) -> "ProteinSet":
        ids = np.asarray(ids, dtype=np.int64)
        lens = self.lengths[ids]
        offs = np.zeros(len(ids) + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        parts = [self.ascii[self.offsets[i]:self.offsets[i + 1]] for i in ids]
        asc = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
        return ProteinSet(asc.astype(np.uint8), offs, self.family[ids].copy(),
                          self.name + f"[subset {len(ids)}]", dict(self.params))


def _substitution_cdf() -> np.ndarray:
    """cdf[a, :] over the 20 standard residues for the replacement of residue a."""
    s = blosum62()[:N_STANDARD, :N_STANDARD].astype(np.float64)
    p = background()
    w = p[None, :] * np.power(2.0, s / 2.0)
    np.fill_diagonal(w, 0.0)
    w /= w.sum(axis=1, keepdims=True)
    return np.cumsum(w, axis=1)


def _draw_background(rng, n, cdf_bg):
    return np.minimum(np.searchsorted(cdf_bg, rng.random(n), side="right"),
                      N_STANDARD - 1).astype(np.uint8)


def _root_lengths(rng, n, lo, hi):
    lens = np.exp(rng.normal(np.log(300.0), 0.6, size=n))
    return np.clip(np.rint(lens), lo, hi).astype(np.int64)


def _zipf_sizes(rng, n_fam, alpha, smax, total):
    """n_fam family sizes ~ Zipf(alpha) truncated to 1..smax, rescaled to sum to total."""
    support = np.arange(1, smax + 1, dtype=np.float64)
    pmf = support ** (-alpha)
    pmf /= pmf.sum()
    sizes = rng.choice(np.arange(1, smax + 1), size=n_fam, p=pmf).astype(np.int64)
    scaled = np.maximum(1, np.floor(sizes * (total / sizes.sum()))).astype(np.int64)
    # hand the remainder (or the excess) out one member at a time, largest first
    order = np.argsort(-scaled, kind="stable")
    k = 0
    while scaled.sum() < total:
        scaled[order[k % n_fam]] += 1
        k += 1
    while scaled.sum() > total:
        idx = order[k % n_fam]
        if scaled[idx] > 1:
            scaled[idx] -= 1
        k += 1
    return scaled


def planted_families(sizes, n_singletons, len_range, seed, p_sub=0.30,
                     indel_rate=0.05 / 3.0, indel_mean=3.0, name="") -> ProteinSet:
    """Families of the given sizes plus unrelated singletons, shuffled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = len_range
    cdf_sub = _substitution_cdf()
    cdf_bg = np.cumsum(background())
    sizes = np.asarray(sizes, dtype=np.int64)
    n_fam = len(sizes)
    root_len = _root_lengths(rng, n_fam, lo, hi)
    seqs, fams = [], []
    for f in range(n_fam):
        root = _draw_background(rng, int(root_len[f]), cdf_bg)
        for _ in range(int(sizes[f])):
            x = root.copy()
            sub = np.flatnonzero(rng.random(x.size) < p_sub)
            if sub.size:
                u = rng.random(sub.size)
                a = x[sub]
                x[sub] = np.minimum((u[:, None] > cdf_sub[a]).sum(axis=1),
                                    N_STANDARD - 1).astype(np.uint8)
            ev = np.flatnonzero(rng.random(x.size) < indel_rate)
            if ev.size:
                ins = rng.random(ev.size) < 0.5
                lens = rng.geometric(1.0 / indel_mean, size=ev.size)
                parts, prev = [], 0
                for p, is_ins, ln in zip(ev.tolist(), ins.tolist(), lens.tolist()):
                    if p < prev:          # inside an earlier deletion
                        continue
                    parts.append(x[prev:p])
                    if is_ins:
                        parts.append(_draw_background(rng, ln, cdf_bg))
                        prev = p
                    else:
                        prev = min(p + ln, x.size)
                parts.append(x[prev:])
                x = np.concatenate(parts)
            if x.size > hi:
                x = x[:hi]
            elif x.size < lo:
                x = np.concatenate([x, _draw_background(rng, lo - x.size, cdf_bg)])
            seqs.append(x)
            fams.append(f)
    single_len = _root_lengths(rng, n_singletons, lo, hi)
    for s in range(n_singletons):
        seqs.append(_draw_background(rng, int(single_len[s]), cdf_bg))
        fams.append(n_fam + s)
    perm = rng.permutation(len(seqs))
    seqs = [seqs[i] for i in perm]
    fam = np.asarray(fams, dtype=np.int32)[perm]
    lens = np.array([s.size for s in seqs], dtype=np.int64)
    offs = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    codes = np.concatenate(seqs) if seqs else np.zeros(0, np.uint8)
    return ProteinSet(_LETTERS[codes].copy(), offs, fam, name,
                      dict(seed=seed, len_range=len_range, n_fam=n_fam,
                           n_singletons=n_singletons))


# ---------------------------------------------------------------------------
# The workloads.  Each is named by what it is; seeds are fixed.
# ---------------------------------------------------------------------------

def families_1k(seed: int = 1) -> ProteinSet:
    """1,000 proteins = 100 families x 10 members, lengths 50-1,000."""
    return planted_families([10] * 100, 0, (50, 1000), seed, name="families_1k")


def zipf_100k(seed: int = 2, n: int = 100_000) -> ProteinSet:
    """100,000 proteins: 10,000 Zipf(1.5, 1-200) families holding 80% of the set,
    plus 20% unrelated singletons; lengths 50-1,000.  ``n`` scales the whole recipe
    (families = n/10) for smaller stand-ins of the same shape."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    n_fam = max(1, n // 10)
    members = int(round(0.8 * n))
    sizes = _zipf_sizes(rng, n_fam, 1.5, 200, members)
    return planted_families(sizes, n - members, (50, 1000), seed, name=f"zipf_{n}")


def zipf_1m(seed: int = 3, n: int = 1_000_000) -> ProteinSet:
    """1,000,000 proteins of the same family recipe, lengths 50-2,000."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    n_fam = max(1, n // 10)
    members = int(round(0.8 * n))
    sizes = _zipf_sizes(rng, n_fam, 1.5, 200, members)
    return planted_families(sizes, n - members, (50, 2000), seed, name=f"zipf1m_{n}")


def random_proteins(n: int, len_range=(50, 1000), seed: int = 0) -> ProteinSet:
    """n unrelated proteins (every one a singleton)."""
    return planted_families([], n, len_range, seed, name=f"random_{n}")


def from_strings(strings, family=None) -> ProteinSet:
    """A set built from explicit letter strings (for hand-made cases)."""
    bs = [s.encode("ascii") for s in strings]
    lens = np.array([len(b) for b in bs], dtype=np.int64)
    offs = np.zeros(len(bs) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    asc = np.frombuffer(b"".join(bs), dtype=np.uint8).copy()
    fam = np.arange(len(bs), dtype=np.int32) if family is None else np.asarray(family, np.int32)
    return ProteinSet(asc, offs, fam, "strings")
