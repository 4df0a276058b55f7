"""The tensor-core (tcgen05, BF16 x BF16 -> FP32) forward convolutions of the
warm-start network: against the FP64 network oracle at base 16 (every
16/32/64-channel layer on tensor cores), and against the CUDA-core BF16 kernels
(to_net_cfg.cuda_cores_only = 1) on the shape the 96x48x48 warm start uses."""
import numpy as np
import pytest

from oracle import net_oracle as N
from tests._util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.mark.parametrize("shape", [(2, 12, 16, 8), (1, 52, 28, 28)])
def test_tc_forward_matches_cuda_core_forward(shape):
    """The same BF16 network with its eligible layers on tensor cores and with
    every layer on CUDA cores (to_net_cfg.cuda_cores_only): same BF16 operands
    per layer, only the FP32 summation order differs."""
    from paper_2005_05436_gb300 import learned as Lr
    r = np.random.default_rng(6)
    x = torch.from_numpy(r.standard_normal(tuple(shape) + (4,)).astype(np.float32)).cuda()
    outs = []
    for tc in (True, False):
        net = Lr.Net(base=16, bf16=True, tensor_cores=tc)
        net.set_params(Lr.he_init(16, seed=5))
        outs.append(net.forward(x).cpu().numpy())
        net.close()
    assert rel(outs[0], outs[1]) <= 1e-2, rel(outs[0], outs[1])
    assert np.abs(outs[0]).max() > 0
