"""Binding checks that run without a GPU: the device-array entry points refuse
host arrays and malformed tensors before the library is called (so no handle
is needed; a valid call would go on to the library)."""
import numpy as np
import pytest

from paper_1911_10274_gb300 import titan as T


def test_set_actuation_dev_refuses_host_and_malformed_arrays_before_the_call():
    torch = pytest.importorskip("torch")
    amp = torch.zeros(6)
    ph = torch.zeros(6)
    with pytest.raises(TypeError, match="CUDA float32"):
        T.titan_set_actuation_dev(0, np.zeros(6, np.float32), ph, 2.0)
    with pytest.raises(TypeError, match="CUDA float32"):
        T.titan_set_actuation_dev(0, amp, ph, 2.0)            # host tensors
    if torch.cuda.is_available():
        d = torch.device("cuda")
        with pytest.raises(TypeError, match="CUDA float32"):
            T.titan_set_actuation_dev(0, torch.zeros(6, dtype=torch.float64, device=d), torch.zeros(6, device=d), 2.0)
        with pytest.raises(ValueError, match="1-D"):
            T.titan_set_actuation_dev(0, torch.zeros(2, 3, device=d), torch.zeros(2, 3, device=d), 2.0)
        with pytest.raises(ValueError, match="same length"):
            T.titan_set_actuation_dev(0, torch.zeros(6, device=d), torch.zeros(5, device=d), 2.0)
