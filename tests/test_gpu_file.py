"""The disk tier of Alg. 8 (gls_solve_file): genotype blocks read from a file
into a ring of pinned slots by a background reader, ahead of the GPU.  The
results must equal gls_solve_stream on the same columns bit for bit (the same
block schedule and kernels), for int8 and 2-bit packed files, with a byte
offset and padded columns, on binary64 and mixed plans (the mixed paths read
int8 slots in place); and the oracle within the path's tolerance.  Missing and
short files give GLS_ERR_IO."""
import numpy as np
import pytest

import oracle
from paper_1210_7325_gb300 import gls, synth
from tests.gpu_util import oracle_ref, relerr

pytestmark = pytest.mark.gpu
IO = 9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1210_7325_gb300 import build
    build.build()


def write_columns(path, cols, ldx, offset):
    """cols: (bytes per column, m) uint8 column-major; padded to ldx, after offset bytes."""
    w, m = cols.shape
    buf = np.full((m, ldx), 0xA5, dtype=np.uint8)   # padding bytes are never read as codes
    buf[:, :w] = cols.T
    with open(path, "wb") as f:
        f.write(b"\x5a" * offset)
        f.write(buf.tobytes())


@pytest.mark.parametrize("prec", ["fp64", "fp16", "bf16"])
@pytest.mark.parametrize("packed,ldx_pad,offset", [(False, 0, 0), (False, 12, 64),
                                                   (True, 0, 0), (True, 5, 3)])
def test_file_equals_stream(tmp_path, prec, packed, ldx_pad, offset):
    import torch
    n = 2100 if prec == "bf16" else 500
    p, m, kmax = 4, 3000, 1024
    pr = synth.problem(n, p, m, 0.5, seed=60 + n, n_markers=max(2 * n, 400))
    X = np.asfortranarray(pr["XR"])
    cols = np.asfortranarray(gls.pack_genotypes(X)) if packed else X.view(np.uint8)
    ldx = cols.shape[0] + ldx_pad
    path = tmp_path / "genotypes.bin"
    write_columns(path, np.asfortranarray(cols), ldx, offset)
    with gls.Plan(n, p, kmax, precision=prec) as plan:
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]), pr["y"])
        Bf = torch.empty((m, p), dtype=torch.float64, pin_memory=True)
        sf = torch.empty(m, dtype=torch.int32, pin_memory=True)
        plan.solve_file(str(path), m, Bf.t(), sf, offset=offset, packed=packed, ldx=ldx)
        src = torch.from_numpy(np.ascontiguousarray(cols.T)).pin_memory()
        Bs = np.zeros((p, m), order="F")
        ss = np.zeros(m, np.int32)
        if packed:
            plan.solve_stream_packed(src.t(), Bs, ss, m=m)
        else:
            plan.solve_stream(src.view(torch.int8).t(), Bs, ss, m=m)
    B = Bf.numpy().T
    assert np.array_equal(B, Bs) and np.array_equal(sf.numpy(), ss)
    tau = oracle.TAU_FP64 if prec == "fp64" else oracle.TAU_MIXED
    Bref, sref = oracle_ref(pr, tau)
    assert np.array_equal(ss, sref)
    assert relerr(B, Bref).max() <= (1e-10 if prec == "fp64" else 1e-6)


def test_file_errors(tmp_path):
    n, p, m = 300, 3, 100
    pr = synth.problem(n, p, m, 0.5, seed=66, n_markers=400)
    path = tmp_path / "short.bin"
    write_columns(path, np.asfortranarray(pr["XR"]).view(np.uint8), n, 0)
    B = np.zeros((p, m + 1), order="F")
    with gls.Plan(n, p, 64, precision="fp16") as plan:
        plan.factor(np.asfortranarray(pr["M"]), np.asfortranarray(pr["XL"]), pr["y"])
        with pytest.raises(gls.GlsError) as ei:
            plan.solve_file(str(tmp_path / "missing.bin"), m, B)
        assert ei.value.status == IO
        with pytest.raises(gls.GlsError) as ei:
            plan.solve_file(str(path), m + 1, B)    # one column more than the file holds
        assert ei.value.status == IO and "fewer than" in str(ei.value)
        plan.solve_file(str(path), m, B[:, :m])     # the plan is still usable
    Bref, _ = oracle_ref(pr, oracle.TAU_MIXED)
    assert relerr(B[:, :m], Bref).max() <= 1e-6
