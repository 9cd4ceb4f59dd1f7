"""Parity of the measurement pre-processing (pat_preprocess, Sec. 4.3) with the FP64
oracle: FP32 transforms on the GPU against FP64 numpy FFTs, relative L2 <= 1e-4 with
eps_rel >= 1e-3.  The regularised filter amplifies the transform's rounding by at most
1 / (2 sqrt(eps_rel)), about 16 here."""
import numpy as np
import pytest

import synthetic as S
from oracle import prep_oracle as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1707_02245_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1707_02245_gb300 import build
    build.build()
    P.load()


def _case(D, T, bipolar, noise, seed):
    det = S.detectors_full_circle(D, 1.2)
    r0, dr = S.radial_sampling(det, T)
    t = r0 + (np.arange(T) + 0.5) * dr
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.6, 2.0, D)
    f = np.exp(-((t[None, :] - centres[:, None]) / 0.1) ** 2)
    xp = (0.07, -0.11)
    p, pcal = S.pressure_measurement(f, det, xp, r0, dr, width=2.5 * dr, noise_level=noise, seed=seed, bipolar=bipolar)
    return det, r0, dr, xp, f, p.astype(np.float32), pcal.astype(np.float32)


@pytest.mark.parametrize("D,T,bipolar,noise,eps", [(8, 300, True, 0.01, 1e-3), (5, 512, False, 0.0, 1e-3),
                                                   (3, 2048, True, 0.02, 1e-2), (2, 1, False, 0.0, 1e-3),
                                                   (16, 129, True, 0.05, 3e-3)])
def test_preprocess_matches_oracle(D, T, bipolar, noise, eps):
    det, r0, dr, xp, f, p, pcal = _case(D, T, bipolar, noise, seed=T + D)
    g = P.Geometry(16, det, T, r0, dr, 32)
    out = torch.empty(D, T, device=DEV)
    P.pat_preprocess(g.handle, torch.from_numpy(p).to(DEV), torch.from_numpy(pcal).to(DEV), xp, eps, out)
    torch.cuda.synchronize()
    ref = R.preprocess(p.astype(np.float64), pcal.astype(np.float64), det, xp, r0, dr, eps)
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-30
    g.close()


def test_preprocess_rejects_bad_arguments():
    det, r0, dr, xp, f, p, pcal = _case(2, 16, True, 0.0, 1)
    g = P.Geometry(8, det, 16, r0, dr, 16)
    pd = torch.from_numpy(p).to(DEV)
    out = torch.empty(2, 16, device=DEV)
    with pytest.raises(P.PatError):
        P.pat_preprocess(g.handle, pd, pd, xp, 0.0, out)
    with pytest.raises(P.PatError):
        P.pat_preprocess(g.handle, pd, pd, tuple(det[0]), 1e-3, out)   # the source on a detector
    g.close()
    g2 = P.Geometry(8, det, 4096, r0, dr / 256, 16)
    big = torch.zeros(2, 4096, device=DEV)
    with pytest.raises(P.PatError):
        P.pat_preprocess(g2.handle, big, big, xp, 1e-3, big)
    g2.close()
