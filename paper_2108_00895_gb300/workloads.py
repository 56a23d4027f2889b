"""Named synthetic workloads shaped like the paper's collections (Sec. 4.1).

Each workload fixes the corpus recipe (sizes, lognormal length mean and clip range,
Zipf exponent), the number of clusters k, the loop limit and the seeds. The paper's
own data (1M tweets, 200k arXiv abstracts) is not available; these seeded corpora
stand in for it. Seeds: corpus 1000 + id, initial documents 2000 + id.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

from . import synth


@dataclass(frozen=True)
class Workload:
    name: str
    n_docs: int
    n_terms: int
    k: int
    nnz_mean: float
    nnz_lo: int
    nnz_hi: int
    zipf_s: float
    max_iter: int
    precision: str          # "fp32" or "bf16" centroid storage for the scoring pass
    prune: str              # "none" or "ncc"
    stop_on_no_change: bool
    seed_id: int

    @property
    def corpus_seed(self) -> int:
        return 1000 + self.seed_id

    @property
    def init_seed(self) -> int:
        return 2000 + self.seed_id

    def corpus(self) -> synth.Csr:
        return synth.make_corpus(self.n_docs, self.n_terms, self.nnz_mean, self.nnz_lo, self.nnz_hi,
                                 self.zipf_s, self.corpus_seed)

    def init_ids(self):
        return synth.init_ids(self.n_docs, self.k, self.init_seed)

    def scaled(self, n_docs: int | None = None, n_terms: int | None = None, k: int | None = None,
               **kw) -> "Workload":
        return replace(self, n_docs=n_docs or self.n_docs, n_terms=n_terms or self.n_terms,
                       k=k or self.k, **kw)

    def describe(self) -> dict:
        return {"workload": self.name, "n_docs": self.n_docs, "n_terms": self.n_terms, "k": self.k,
                "nnz": f"lognormal(mean {self.nnz_mean:g}) clipped to [{self.nnz_lo},{self.nnz_hi}]",
                "terms": f"Zipf(s={self.zipf_s:g}) without replacement",
                "values": "(Poisson(1)+1)*ln(N/df), L2-normalised",
                "precision": self.precision, "prune": self.prune, "max_iter": self.max_iter,
                "seeds": {"corpus": self.corpus_seed, "init": self.init_seed}}


# Plain exact spherical k-means, FP32, 20 Lloyd iterations.
SMALL = Workload("plain-fp32 N=2000 d=5000 k=20", 2000, 5000, 20, 60.0, 5, 400, 1.1, 20,
                 "fp32", "none", False, 1)
# Full vs pruned assignment, FP32, up to 50 iterations or no assignment change.
MEDIUM = Workload("ncc-fp32 N=300000 d=100000 k=1000", 300_000, 100_000, 1000, 120.0, 5, 2000, 1.05,
                  50, "fp32", "ncc", True, 2)
# Precision form: BF16 centroids, FP32 accumulation, FP64 rescoring, up to 30 iterations.
LARGE = Workload("ncc-bf16 N=2000000 d=250000 k=10000", 2_000_000, 250_000, 10_000, 150.0, 5, 2000,
                 1.05, 30, "bf16", "ncc", True, 3)

ALL = {"small": SMALL, "medium": MEDIUM, "large": LARGE}
