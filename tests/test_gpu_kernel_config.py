"""Launch configuration of the persistent kernel on the GPU. The FP64
instance (plans whose products are all FP64, no tensor-core code) keeps two
resident CTAs per SM at the shared memory its launches ask for: the FP64
throughput and the schedule assume it. The instance with tensor-core parts
uses tcgen05 instructions, and a kernel that does runs at most one CTA per
SM on this driver (any tcgen05 instruction, whatever tensor memory it
allocates), which the occupancy query must report as such."""
import pytest

from tests.gpu_helpers import need_gpu


@pytest.mark.gpu
def test_fp64_instance_two_resident_ctas_per_sm():
    S = need_gpu()
    assert S.stiles_debug_occupancy(False) == 2


@pytest.mark.gpu
def test_tensor_instance_is_resident():
    S = need_gpu()
    assert S.stiles_debug_occupancy(True) >= 1
