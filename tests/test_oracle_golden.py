"""The frozen oracle output of tests/golden (written by make_golden.py, which
calls only the oracle) guards the oracle's arithmetic against unintended
change; the FP64 GPU path is compared with the stored values as well."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_q_n8_two_stream.txt")
GOLD_VHS = os.path.join(HERE, "golden", "oracle_q_vhs_alpha0_n8_two_stream.txt")


def load(path=GOLD):
    case, arrays = {}, {}
    for line in open(path):
        if line.startswith("#"):
            case = dict(kv.split("=") for kv in line[1:].split())
        else:
            name, *vals = line.split()
            arrays[name] = np.array([float(v) for v in vals]).reshape(8, 8, 8)
    return case, arrays["f"], arrays["Q"]


def test_oracle_reproduces_the_frozen_output(oracle):
    case, f, Q = load()
    tab = oracle.tables(int(case["n"]), float(case["L"]), int(case["ktype"]), float(case["C"]),
                        int(case["A1"]), int(case["A2"]), int(case["rule"]))
    got = oracle.collide(f[None], tab, kn=float(case["kn"]), project=True)[0]
    assert np.linalg.norm(got - Q) <= 1e-13 * np.linalg.norm(Q)


def test_stored_input_is_the_seeded_input():
    from paper_1701_01608_gb300 import inputs as I
    case, f, _ = load()
    g = I.two_stream((1, 1, 1), int(case["n"]), float(case["L"]), seed=int(case["seed"]),
                     noise=float(case["noise"]))[0]
    # to the last bits of the platform's exp (the stored file was written on x86-64)
    assert np.allclose(g, f, rtol=1e-14, atol=0.0)


@pytest.mark.gpu
def test_fp64_gpu_matches_the_frozen_output():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    case, f, Q = load()
    ctx = fks.Context(fks.Config(ncell=(1, 1, 1), n=8, L=float(case["L"]), kernel=int(case["ktype"]),
                                 C=float(case["C"]), kn=float(case["kn"]), A1=int(case["A1"]), A2=int(case["A2"]),
                                 rule=int(case["rule"]), precision=fks.FKS_FP64))
    fd = torch.from_numpy(f[None].copy()).cuda()
    out = torch.empty_like(fd)
    ctx.collide(fd, out)
    got = out[0].cpu().numpy()
    assert np.linalg.norm(got - Q) <= 1e-10 * np.linalg.norm(Q)


def test_oracle_reproduces_the_frozen_vhs_output(oracle):
    case, f, Q = load(GOLD_VHS)
    got = oracle.collide_vhs(f[None], int(case["n"]), float(case["L"]), float(case["alpha"]), float(case["C"]),
                             int(case["A1"]), int(case["A2"]), int(case["rule"]), kn=float(case["kn"]),
                             project=True)[0]
    assert np.linalg.norm(got - Q) <= 1e-13 * np.linalg.norm(Q)


@pytest.mark.gpu
def test_fp64_gpu_vhs_matches_the_frozen_output():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    case, f, Q = load(GOLD_VHS)
    ctx = fks.Context(fks.Config(ncell=(1, 1, 1), n=8, L=float(case["L"]), kernel=fks.VHS, alpha=float(case["alpha"]),
                                 C=float(case["C"]), kn=float(case["kn"]), A1=int(case["A1"]), A2=int(case["A2"]),
                                 rule=int(case["rule"]), precision=fks.FKS_FP64))
    fd = torch.from_numpy(f[None].copy()).cuda()
    out = torch.empty_like(fd)
    ctx.collide(fd, out)
    assert np.linalg.norm(out[0].cpu().numpy() - Q) <= 1e-10 * np.linalg.norm(Q)
