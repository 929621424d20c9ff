"""Seeded synthetic inputs shaped like the paper's GWAS workloads.

This module only draws inputs (M, X_L, y, X_R); it holds none of the GLS
arithmetic, so both the GPU path's tests/benchmarks and the CPU oracle can be
fed from it.

Recipe (the paper fixes only shapes and SPD-ness of M; the rest is the stated
synthetic workload):
  * kinship: G is n x n_markers with column j ~ Binomial(2, f_j),
    f_j ~ U(0.05, 0.5); columns standardized by their empirical mean and
    (population) standard deviation, zero-variance columns redrawn;
    K = G G^T / n_markers; Phi_ij = K_ij / sqrt(K_ii K_jj) (unit diagonal);
    M = h Phi + (1 - h) I, SPD for 0 <= h < 1.
  * covariates: X_L = [1, N(0,1), ..., N(0,1)], n x (p - 1).
  * phenotype: y ~ N(0, 1), n.
  * genotypes: X_R is n x m int8, SNP i ~ Binomial(2, f_i), f_i ~ U(0.05, 0.5),
    stored column-major (each SNP's n genotypes contiguous).
Every draw comes from a counter-based Philox stream keyed by (seed, stream id).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20121030

_STREAM_KINSHIP = 1
_STREAM_COVARIATES = 2
_STREAM_PHENOTYPE = 3
_STREAM_GENOTYPES = 4


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream)])))


def kinship_markers(n: int, seed: int, n_markers: int = 5000) -> np.ndarray:
    """Standardized marker matrix G (n x n_markers, float64, C order)."""
    if n < 2:
        raise ValueError("a marker column needs n >= 2 individuals to have variance")
    g = rng(seed, _STREAM_KINSHIP)
    f = g.uniform(0.05, 0.5, size=n_markers)
    G = g.binomial(2, f[None, :], size=(n, n_markers)).astype(np.float64)
    for _ in range(10000):
        sd = G.std(axis=0)
        bad = np.flatnonzero(sd == 0.0)
        if bad.size == 0:
            break
        fb = g.uniform(0.05, 0.5, size=bad.size)
        G[:, bad] = g.binomial(2, fb[None, :], size=(n, bad.size))
    else:
        raise RuntimeError("could not draw polymorphic marker columns")
    G -= G.mean(axis=0)
    G /= G.std(axis=0)
    return G


def kinship_M(n: int, h: float, seed: int, n_markers: int = 5000, device: str = "cpu"):
    """M = h Phi + (1 - h) I as an n x n float64 array (symmetric, so C order
    equals column-major).  ``device`` selects where G G^T is multiplied
    (a torch device string); the result is always returned on the host."""
    if n == 1:  # Phi has unit diagonal, so M = h + (1 - h) = 1
        return np.ones((1, 1))
    G = kinship_markers(n, seed, n_markers)
    if device == "cpu":
        K = (G @ G.T) / n_markers
    else:
        import torch
        Gt = torch.from_numpy(G).to(device)
        K = (Gt @ Gt.T).div_(n_markers).cpu().numpy()
    d = np.sqrt(np.diag(K).copy())
    Phi = K / d[:, None] / d[None, :]
    Phi = 0.5 * (Phi + Phi.T)
    np.fill_diagonal(Phi, 1.0)
    M = h * Phi
    M[np.diag_indices(n)] += (1.0 - h)
    return np.ascontiguousarray(M)


def kinship_M_torch(n: int, h: float, seed: int, n_markers: int = 5000, device="cuda"):
    """The kinship recipe above drawn with torch on ``device`` and multiplied in
    FP32 (fast enough to generate one M per request at serving rates).  The
    marker draws use torch's generator, so the matrix differs from
    ``kinship_M`` for the same seed.  Returns an (n, n) float64 tensor
    (symmetric, so row- and column-major storage coincide)."""
    M = kinship_phi_torch(n, seed, n_markers, device)
    M.mul_(h)
    M.diagonal().add_(1.0 - h)
    return M


def kinship_phi_torch(n: int, seed: int, n_markers: int = 5000, device="cuda"):
    """Phi (unit diagonal, n x n float64 tensor) of the kinship recipe, drawn
    with torch on ``device`` (see kinship_M_torch)."""
    import torch
    dev = torch.device(device)
    if n < 2:  # one sample: Phi = [1]
        return torch.ones((n, n), dtype=torch.float64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 1000003 + _STREAM_KINSHIP)
    f = torch.rand(n_markers, generator=gen, device=dev) * 0.45 + 0.05

    def draw(fcols):
        # Binomial(2, f) from one uniform: [u >= (1-f)^2] + [u >= 1 - f^2]
        u = torch.rand((n, fcols.numel()), generator=gen, device=dev)
        return (u >= (1.0 - fcols) * (1.0 - fcols)).float() + (u >= 1.0 - fcols * fcols).float()

    G = draw(f)
    for _ in range(10000):
        bad = torch.nonzero(G.std(dim=0, unbiased=False) == 0).flatten()
        if bad.numel() == 0:
            break
        fb = torch.rand(bad.numel(), generator=gen, device=dev) * 0.45 + 0.05
        G[:, bad] = draw(fb)
    G = (G - G.mean(dim=0)) / G.std(dim=0, unbiased=False)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        K = (G @ G.T) / n_markers
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    d = torch.sqrt(torch.diagonal(K))
    Phi = (K / d[:, None] / d[None, :]).double()
    Phi = 0.5 * (Phi + Phi.T)
    Phi.fill_diagonal_(1.0)
    return Phi


def covariates(n: int, p: int, seed: int) -> np.ndarray:
    """X_L (n x (p-1)) column-major: a column of ones then N(0,1) columns."""
    if p < 1:
        raise ValueError("p >= 1")
    g = rng(seed, _STREAM_COVARIATES)
    XL = np.empty((n, max(p - 1, 0)), dtype=np.float64, order="F")
    if p >= 2:
        XL[:, 0] = 1.0
        for c in range(1, p - 1):
            XL[:, c] = g.standard_normal(n)
    return XL


def phenotype(n: int, seed: int) -> np.ndarray:
    return rng(seed, _STREAM_PHENOTYPE).standard_normal(n)


def genotypes_np(n: int, m: int, seed: int) -> np.ndarray:
    """X_R (n x m int8, column-major) on the host with numpy; for small m."""
    g = rng(seed, _STREAM_GENOTYPES)
    f = g.uniform(0.05, 0.5, size=m)
    X = np.empty((n, m), dtype=np.int8, order="F")
    for i in range(m):
        X[:, i] = g.binomial(2, f[i], size=n)
    return X


def genotypes_torch(n: int, m: int, seed: int, device="cpu", chunk: int = 8192, out=None):
    """X_R as a torch int8 tensor of shape (m, n) (row i = SNP i, i.e. the
    column-major n x m matrix), drawn on ``device`` in chunks of SNPs.
    Binomial(2, f) is drawn from one uniform u per genotype by its inverse
    distribution function: x = [u >= (1-f)^2] + [u >= 1 - f^2], so that
    P(0) = (1-f)^2, P(1) = 2 f (1-f) and P(2) = f^2."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 1000003 + _STREAM_GENOTYPES)
    if out is None:
        out = torch.empty((m, n), dtype=torch.int8, device=dev)
    for s in range(0, m, chunk):
        c = min(chunk, m - s)
        f = torch.rand((c, 1), generator=gen, device=dev, dtype=torch.float32) * 0.45 + 0.05
        u = torch.rand((c, n), generator=gen, device=dev, dtype=torch.float32)
        x = (u >= (1.0 - f) * (1.0 - f)).to(torch.int8)
        x += u >= 1.0 - f * f
        out[s:s + c].copy_(x)
    return out


def problem(n: int, p: int, m: int, h: float, seed: int, n_markers: int = 5000,
            kin_device: str = "cpu"):
    """A small complete problem on the host: dict(M, XL, y, XR) with XR n x m int8."""
    return dict(
        M=kinship_M(n, h, seed, n_markers, device=kin_device),
        XL=covariates(n, p, seed),
        y=phenotype(n, seed),
        XR=genotypes_np(n, m, seed),
    )


_STREAM_BANK = 5


class ServingBank:
    """Request inputs for a serving run, drawn once before the requests arrive
    so that admitting a request costs a slice and one elementwise kernel, not
    a fresh synthesis (which would make the measured latency that of the input
    generator rather than of the server).

    Two device-resident banks, for N = the largest n of the stream:
      * Phi_bank: the kinship recipe's Phi for N individuals (N x N float64);
      * X_bank: m_max SNPs of N individuals (m_max x N int8, SNP-major),
        SNP i ~ Binomial(2, f_i), f_i ~ U(0.05, 0.5).
    Request (n, p, m, h) with seed s draws offsets o ~ U{0..N-n} and
    c ~ U{0..m_max-m} from s; then
      M   = h Phi_bank[o:o+n, o:o+n] + (1 - h) I  (a principal submatrix of a
            correlation matrix: unit diagonal and SPD, so M is SPD for h < 1),
      X_R = X_bank[c:c+m, o:o+n]^T  (column-major n x m view, leading dim N),
      X_L = covariates(n, p, s), y = phenotype(n, y_seed).
    Equal seeds give equal (M, X_L, X_R), so a request that repeats an earlier
    scan with a new phenotype sees the same factor inputs."""

    def __init__(self, n_max: int, m_max: int, seed: int, n_markers: int = 5000,
                 device="cuda"):
        import torch
        self.N, self.m_max = int(n_max), int(m_max)
        self.device = torch.device(device)
        self.phi = kinship_phi_torch(self.N, seed, n_markers, device)
        self.X = genotypes_torch(self.N, self.m_max, seed + 1, device=device)

    def offsets(self, n: int, m: int, seed: int):
        g = rng(seed, _STREAM_BANK)
        o = int(g.integers(0, self.N - n + 1))
        c = int(g.integers(0, self.m_max - m + 1))
        return o, c

    def request(self, n: int, p: int, m: int, h: float, seed: int, y_seed: int,
                with_factor_inputs: bool = True):
        """(M, X_L, y, X_R) as device tensors (M, X_L None without factor inputs)."""
        import torch
        if n > self.N or m > self.m_max:
            raise ValueError(f"request n={n}, m={m} exceeds the bank ({self.N}, {self.m_max})")
        o, c = self.offsets(n, m, seed)
        M = XL = None
        if with_factor_inputs:
            M = self.phi[o:o + n, o:o + n] * h
            M.diagonal().add_(1.0 - h)
            M = M.t()  # exactly symmetric: the column-major view of the same matrix
            if p > 1:
                XL = torch.from_numpy(np.ascontiguousarray(covariates(n, p, seed).T))
                XL = XL.to(self.device).t()
        y = torch.from_numpy(phenotype(n, y_seed)).to(self.device)
        XR = self.X[c:c + m, o:o + n]  # (m, n) view: X_R^T, row stride N
        return M, XL, y, XR
