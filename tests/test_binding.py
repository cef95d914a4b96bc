"""Host-side argument checks of the Python binding (no GPU needed)."""
import pytest


def test_batch_size_is_checked_before_any_call():
    from paper_2404_09758_gb300 import Batch
    with pytest.raises(ValueError):
        Batch([])
    with pytest.raises(ValueError):
        Batch([None] * 65)
