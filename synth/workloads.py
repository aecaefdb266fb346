"""The five Lloyd k-means workloads, as shapes and mixture parameters.

Each single-instance workload draws n points from an isotropic Gaussian mixture
with m components (means uniform in [-R, R]^d, standard deviation sigma, equal
weights), starts from C0 = the first k points, and runs a fixed number of Lloyd
iterations (tol = 0). Seeds are 0x5EED0000 + index.
"""
from __future__ import annotations

from dataclasses import dataclass, field

SEED_BASE = 0x5EED0000


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    k: int
    m: int
    R: float
    sigma: float
    iters: int
    precision: tuple = ("fp32",)
    seed: int = 0
    instances: int = 1
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def flops_per_iter(self) -> float:
        """Algorithmic distance FLOPs of one Lloyd iteration: 2*n*k*d (the contraction only)."""
        return 2.0 * self.n * self.k * self.d


WORKLOADS = {
    "plain_n10k_d16_k8": Workload(
        "plain_n10k_d16_k8", n=10_000, d=16, k=8, m=8, R=10.0, sigma=1.0, iters=10,
        precision=("fp32",), seed=SEED_BASE + 0,
        note="small plain k-means; lowest-index ties"),
    "fp32_n1M_d64_k256": Workload(
        "fp32_n1M_d64_k256", n=1 << 20, d=64, k=256, m=256, R=20.0, sigma=1.0, iters=20,
        precision=("fp32",), seed=SEED_BASE + 1,
        note="plain FP32 fused Lloyd step"),
    "prec_n4M_d128_k1024": Workload(
        "prec_n4M_d128_k1024", n=1 << 22, d=128, k=1024, m=1024, R=20.0, sigma=1.0, iters=20,
        precision=("fp32", "bf16", "fp8"), seed=SEED_BASE + 2,
        note="BF16 and FP8-E4M3 distance + FP32 recheck vs plain FP32"),
    "batched_512": Workload(
        "batched_512", n=0, d=0, k=0, m=0, R=10.0, sigma=1.0, iters=15,
        precision=("bf16",), seed=SEED_BASE + 3, instances=512,
        note="512 instances; n log-uniform [1e3,2e5], d in {8,32,64,128}, k log-uniform [4,512]"),
    "large_n8M_d256_k8192": Workload(
        "large_n8M_d256_k8192", n=1 << 23, d=256, k=8192, m=8192, R=5.0, sigma=0.5, iters=10,
        precision=("fp8",), seed=SEED_BASE + 4,
        note="FP8-E4M3 distance + FP32 recheck; frequent near-ties"),
}


def batched_instances(w: Workload = WORKLOADS["batched_512"]):
    """The per-instance workloads of the batched set: instance b uses seed base+b, m = k."""
    from . import instance_shape

    out = []
    for b in range(w.instances):
        seed = w.seed * 1000 + b
        n, d, k = instance_shape(seed)
        out.append(Workload(f"{w.name}[{b}]", n=n, d=d, k=k, m=k, R=w.R, sigma=w.sigma,
                            iters=w.iters, precision=w.precision, seed=seed))
    return out


@dataclass(frozen=True)
class SpadeWorkload:
    """SPADE downsampling input (Sec. 4.1): n rows of a Gaussian mixture (cell
    populations) with the two widths the paper's generated code prints. The
    paper gives neither d nor the data; sigma is chosen so that apprx_width is
    about 1.5 x the median nearest-neighbour L1 distance of a row."""
    name: str
    n: int
    d: int
    m: int
    R: float
    sigma: float
    apprx: float
    kernel: float
    seed: int
    note: str = ""


SPADE_WORKLOADS = {
    "spade_n235k_d16": SpadeWorkload(
        "spade_n235k_d16", n=235_000, d=16, m=40, R=10.0, sigma=0.55,
        apprx=6.689027961, kernel=22.29675987, seed=SEED_BASE + 0x200,
        note="row length 235,000 as in the paper's typical dataset; widths as printed in its generated code"),
}
