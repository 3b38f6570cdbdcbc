"""The binary32 noise's quotient and square root (section 2, eq. (Papos2):
the specification rounds both correctly) are short sequences on the GPU;
they must equal the IEEE operations on every binary32 input the noise can
give them (cf_noise_selfcheck enumerates both domains), and the draws must
stay bit-exact against the oracle (tests/test_gpu_parity.py)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1406_6072_gb300 import cf  # noqa: E402


def test_noise_quotient_and_square_root_round_correctly_on_their_domains():
    mism, examples = cf.cf_noise_selfcheck()
    assert mism == (0, 0), "first mismatching inputs (bits): m %#010x, x %#010x" % examples
