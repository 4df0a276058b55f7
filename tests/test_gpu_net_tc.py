"""The tensor-core (tcgen05, BF16 x BF16 -> FP32) forward convolutions of the
warm-start network: against the FP64 network oracle at base 16 (every
16/32/64-channel layer on tensor cores), and against the CUDA-core BF16 kernels
(TOPO_NET_TC=0, read once per process, hence the subprocess) on the shape the
96x48x48 warm start uses."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import net_oracle as N
from tests._util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2005_05436_gb300 import build
    build.build()


def test_tc_forward_matches_oracle_base16():
    from paper_2005_05436_gb300.learned import Net
    base = 16
    r = np.random.default_rng(3)
    theta = N.init_params(base, seed=3) + 0.02 * r.standard_normal(N.n_params(base))
    x = r.standard_normal((8, 12, 8, 4))
    net = Net(base=base, bf16=True)
    net.set_params(theta.astype(np.float32))
    y = net.forward(torch.from_numpy(x[None]).float().cuda()).cpu().numpy()[0]
    y_ref, _ = N.forward(theta.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64), base)
    assert rel(y, y_ref) <= 3e-2, rel(y, y_ref)


SCRIPT = r'''
import sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2005_05436_gb300 import learned as Lr
net = Lr.Net(base=16, bf16=True)
net.set_params(Lr.he_init(16, seed=5))
r = np.random.default_rng(6)
x = torch.from_numpy(r.standard_normal({shape} + (4,)).astype(np.float32)).cuda()
np.save({out!r}, net.forward(x).cpu().numpy())
'''


@pytest.mark.parametrize("shape", [(2, 12, 16, 8), (1, 52, 28, 28)])
def test_tc_forward_matches_cuda_core_forward(tmp_path, shape):
    outs = []
    for tc in ("1", "0"):
        out = str(tmp_path / f"y_{tc}.npy")
        env = dict(os.environ, TOPO_NET_TC=tc)
        res = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, shape=tuple(shape), out=out)],
                             env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert res.returncode == 0, res.stderr[-3000:]
        outs.append(np.load(out))
    # same BF16 operands per layer; only the FP32 summation order differs
    assert rel(outs[0], outs[1]) <= 1e-2, rel(outs[0], outs[1])
    assert np.abs(outs[0]).max() > 0
