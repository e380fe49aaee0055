"""One image in tiles with a halo on the GPU (denoise_bm3d_tiled): every
kernel is deterministic and the aggregation sums are exact, so with the halo
of dn_bm3d_halo the tiled result equals denoise_bm3d on the whole image bit
for bit -- grey and colour, ragged edge tiles, batched tiles of equal
extent, the high-noise first pass, and a 2048 x 1536 image."""
import numpy as np
import pytest

from gpu_util import dev, host, need_gpu
from paper_2403_03488_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("C,H,W,sigma,tile,batch", [(1, 333, 517, 25.0, 120, 4), (3, 300, 420, 25.0, 128, 2),
                                                   (1, 400, 400, 50.0, 160, 3), (1, 96, 80, 15.0, 256, 1),
                                                   (1, 270, 270, 25.0, 90, 9)])
def test_tiled_equals_whole_image(C, H, W, sigma, tile, batch):
    from paper_2403_03488_gb300 import api
    _, noisy = synth.make_batch([150], H, W, sigma, C=C)
    x = dev(noisy)
    whole = host(api.denoise_bm3d(x, sigma))[0]
    tiled = host(api.denoise_bm3d_tiled(x[0].contiguous(), sigma, tile=tile, max_batch=batch))
    np.testing.assert_array_equal(tiled, whole)
    assert api.device_error() == 0


def test_tiled_full_size():
    """A 2048 x 1536 grey image (the paper's larger test images are 1600 x 1200
    and 4048 x 3044) in 512-pixel tiles: bit-identical to the whole image."""
    from paper_2403_03488_gb300 import api
    clean, noisy = synth.make_batch([151], 1536, 2048, 25.0)
    x = dev(noisy)
    whole = host(api.denoise_bm3d(x, 25.0))[0]
    tiled = host(api.denoise_bm3d_tiled(x[0].contiguous(), 25.0, tile=512, max_batch=6))
    np.testing.assert_array_equal(tiled, whole)
