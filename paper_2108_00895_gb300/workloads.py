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
    shift_tol: float = -1.0     # Sec. 4.1 stop rule (max squared centroid shift); < 0: off

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
                "shift_tol": self.shift_tol,
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

# Analogs of the paper's two collections (Sec. 4.1): 1M tweets (783,304 terms, 10 nonzeros
# on average) and 200k abstracts (325,556 terms, 58 on average), clustered with the paper's
# stop rule (no assignment change or max squared centroid shift < 1e-4) at k = 50, 500 or
# 5000 (Table 1). FP32 centroids with FP64 rescoring: exact, like the paper's CPU method.
TWEETS = Workload("tweets-like N=1000000 d=783304 k=5000", 1_000_000, 783_304, 5000, 10.0, 2, 60, 1.05,
                  200, "fp32", "ncc", True, 6, 1e-4)
ABSTRACTS = Workload("abstracts-like N=200000 d=325556 k=5000", 200_000, 325_556, 5000, 58.0, 5, 600, 1.05,
                     200, "fp32", "ncc", True, 7, 1e-4)

ALL = {"small": SMALL, "medium": MEDIUM, "large": LARGE, "tweets": TWEETS, "abstracts": ABSTRACTS}


@dataclass(frozen=True)
class BatchedWorkload:
    """Many independent clustering instances of different sizes (the batched form): per
    instance N log-uniform in [n_lo, n_hi], d uniform over `vocab`, k log-uniform in
    [k_lo, k_hi] (and at most N), lognormal(nnz_mean) lengths clipped to [5, 2000], Zipf terms,
    FP32 centroids, a fixed number of Lloyd steps."""
    name: str
    n_instances: int
    n_lo: int
    n_hi: int
    vocab: tuple
    k_lo: int
    k_hi: int
    nnz_mean: float
    zipf_s: float
    max_iter: int
    seed: int

    def specs(self):
        import math
        u = synth.uniform(self.seed, 1, 3 * self.n_instances)
        out = []
        for q in range(self.n_instances):
            n = int(round(math.exp(math.log(self.n_lo) + u[3 * q] * (math.log(self.n_hi) - math.log(self.n_lo)))))
            d = int(self.vocab[min(len(self.vocab) - 1, int(u[3 * q + 1] * len(self.vocab)))])
            k = int(round(math.exp(math.log(self.k_lo) + u[3 * q + 2] * (math.log(self.k_hi) - math.log(self.k_lo)))))
            out.append((n, d, min(k, n)))
        return out

    def instances(self):
        """[(corpus, k, initial ids)] with seeds derived from the instance index."""
        res = []
        for q, (n, d, k) in enumerate(self.specs()):
            docs = synth.make_corpus(n, d, self.nnz_mean, 5, 2000, self.zipf_s, self.seed * 1000 + q)
            res.append((docs, k, synth.init_ids(n, k, self.seed * 1000 + 500 + q)))
        return res

    def describe(self) -> dict:
        return {"workload": self.name, "instances": self.n_instances,
                "n_docs": f"log-uniform [{self.n_lo}, {self.n_hi}]", "n_terms": list(self.vocab),
                "k": f"log-uniform [{self.k_lo}, {self.k_hi}]",
                "nnz": f"lognormal(mean {self.nnz_mean:g}) clipped to [5,2000]",
                "terms": f"Zipf(s={self.zipf_s:g}) without replacement", "precision": "fp32",
                "max_iter": self.max_iter, "seed": self.seed}


# Batched form: 256 uneven instances, 20 Lloyd steps each, FP32.
BATCHED = BatchedWorkload("batched-fp32 256 instances", 256, 1000, 200_000, (20_000, 50_000, 100_000), 16, 2048,
                          80.0, 1.1, 20, 4)


@dataclass(frozen=True)
class ServingWorkload:
    """Serving form: a resident BF16 centroid set (k, d) under a device budget; Poisson
    arrivals at `rate` per second, a fraction `p_assign` of them assignment requests of
    log-uniform [1, assign_hi] new documents (drawn from a pool of documents like the large
    workload's), the rest clustering jobs of log-uniform N in [job_n_lo, job_n_hi] and k in
    [job_k_lo, job_k_hi] for `job_iters` steps."""
    name: str
    k: int
    n_terms: int
    budget_gb: float
    rate: float
    p_assign: float
    assign_hi: int
    job_n_lo: int
    job_n_hi: int
    job_k_lo: int
    job_k_hi: int
    job_iters: int
    pool_docs: int
    nnz_mean: float
    zipf_s: float
    seed: int

    def pool(self):
        return synth.make_corpus(self.pool_docs, self.n_terms, self.nnz_mean, 5, 2000, self.zipf_s, 1000 + self.seed)

    def describe(self) -> dict:
        return {"workload": self.name, "k": self.k, "n_terms": self.n_terms, "budget_GB": self.budget_gb,
                "rate_per_s": self.rate, "assign_fraction": self.p_assign,
                "assign_docs": f"log-uniform [1, {self.assign_hi}]",
                "job_n": f"log-uniform [{self.job_n_lo}, {self.job_n_hi}]",
                "job_k": f"log-uniform [{self.job_k_lo}, {self.job_k_hi}]", "job_iters": self.job_iters,
                "documents": f"lognormal(mean {self.nnz_mean:g}) clipped to [5,2000], Zipf(s={self.zipf_s:g}), "
                             f"pool of {self.pool_docs} seeded documents"}


SERVING = ServingWorkload("serving bf16 k=10000 d=250000", 10_000, 250_000, 40.0, 2000.0, 0.9, 4096,
                          10_000, 500_000, 64, 4096, 20, 500_000, 150.0, 1.05, 5)
