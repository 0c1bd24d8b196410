"""The device copy of the seeded generator (libhuffsynth.so) draws exactly
what synth.py draws, so inputs made on the GPU can be regenerated for the
oracle on the host."""
import numpy as np
import pytest

from paper_2010_10039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width", [1, 2, 4])
def test_device_draw_equals_host_draw(width):
    K = {1: 256, 2: 1024, 4: 1024}[width]
    table = synth.cdf_table(synth.laplace_pmf(K, K // 2, 3.0))
    host = synth.draw(7, 3, 300_001, table, width)
    dev = synth.draw_device(7, 3, 300_001, table, width).cpu().numpy().view(host.dtype)
    assert np.array_equal(dev, host)


def test_device_draw_with_mapping_large_table_and_offset():
    K = 65536
    table = synth.cdf_table(synth.zipf_pmf(K, 1.1))
    perm = synth.permutation(3, K)
    host = synth.draw(3, 0, 200_000, table, 4, mapping=perm)
    dev = synth.draw_device(3, 0, 150_000, table, 4, mapping=perm, start=50_000).cpu().numpy().view(np.uint32)
    assert np.array_equal(dev, host[50_000:])


def test_device_draw_of_a_batched_field():
    n, b = synth.batch_field_params(5)
    host = synth.batch_field(5)
    dev = synth.draw_device(4, 5, n, synth.cdf_table(synth.laplace_pmf(1024, 512, b)), 2)
    assert np.array_equal(dev.cpu().numpy().view(np.uint16), host)
