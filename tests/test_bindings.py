"""The Python binding's own checks of the buffers it passes to the C ABI
(the library sees plain pointers, so sizes are checked above it).  Runs on
the CPU: every call below fails a check while its arguments are evaluated,
before the library function is entered, so no pointer of a stand-in object
ever reaches the library."""
import pytest

torch = pytest.importorskip("torch")

import paper_1710_10096_gb300 as sff


class FakeCuda:
    """Stands in for a CUDA tensor of `nbytes` bytes (shape / strides for images)."""
    is_cuda = True

    def __init__(self, nbytes, contiguous=True, shape=None, strides=None):
        self._n, self._c = nbytes, contiguous
        self.shape = shape if shape is not None else (nbytes,)
        self._strides = strides

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def element_size(self):
        return 1

    def dim(self):
        return len(self.shape)

    def stride(self, k):
        return self._strides[k]

    def data_ptr(self):
        return 1 << 20


@pytest.fixture(scope="module", autouse=True)
def built():
    sff.build()


def test_cpu_tensors_are_rejected():
    img = torch.zeros((48, 64, 3), dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        sff.sgm(img, img, torch.empty((48, 64), dtype=torch.int16), torch.empty(1 << 20, dtype=torch.uint8))
    with pytest.raises(ValueError, match="CUDA"):
        sff.interpolate(torch.empty(20 * 8, dtype=torch.uint8), torch.zeros(1, dtype=torch.int32), 8, 64, 48,
                        sff.default_interp_params(64, 48, 700.0, 0.5), torch.empty((48, 64, 4)),
                        torch.empty(1 << 20, dtype=torch.uint8))


def test_small_buffers_are_rejected():
    w, h = 64, 48
    p = sff.default_params()
    pb = sff.pyramid_bytes(w, h, p)
    ok_pyr = FakeCuda(pb)
    with pytest.raises(ValueError, match="pyramid"):
        sff.match_views(ok_pyr, ok_pyr, FakeCuda(pb - 1), ok_pyr, w, h, 0, 1, FakeCuda(8 * w * h),
                        FakeCuda(4 * w * h), FakeCuda(1 << 20), p)
    with pytest.raises(ValueError, match="cost"):
        sff.match_views(ok_pyr, ok_pyr, ok_pyr, ok_pyr, w, h, 0, 1, FakeCuda(8 * w * h), FakeCuda(4 * w * h - 4),
                        FakeCuda(1 << 20), p)
    with pytest.raises(ValueError, match="field"):
        sff.interpolate(FakeCuda(20 * 8), FakeCuda(4), 8, w, h, sff.default_interp_params(w, h, 700.0, 0.5),
                        FakeCuda(16 * w * h - 1), FakeCuda(1 << 20))
    with pytest.raises(ValueError, match="seeds"):
        sff.emit_seeds(FakeCuda(8 * w * h, shape=(h, w, 4)), FakeCuda(4 * w * h), FakeCuda(w * h), FakeCuda(w * h),
                       FakeCuda(20 * 100 - 1), 100, FakeCuda(4), FakeCuda(1 << 20))
    with pytest.raises(ValueError, match="phi"):
        sff.match_views_sift(ok_pyr, ok_pyr, ok_pyr, ok_pyr, FakeCuda(16 * p.num_scales * w * h),
                             FakeCuda(16 * p.num_scales * w * h - 16), FakeCuda(16 * p.num_scales * w * h),
                             FakeCuda(16 * p.num_scales * w * h), w, h, 0, 1, FakeCuda(8 * w * h),
                             FakeCuda(4 * w * h), FakeCuda(1 << 20), p)


def test_strided_buffers_and_images_are_rejected():
    w, h = 64, 48
    with pytest.raises(ValueError, match="contiguous"):
        sff.consistency_filter(FakeCuda(8 * w * h, shape=(h, w, 4)), FakeCuda(4 * w * h), FakeCuda(8 * w * h),
                               FakeCuda(4 * w * h), FakeCuda(w * h, contiguous=False), FakeCuda(w * h),
                               FakeCuda(1 << 20))
    # planar (channel-major) and row-overlapping images
    planar = FakeCuda(3 * w * h, shape=(h, w, 3), strides=(w, 1, w * h))
    overlap = FakeCuda(3 * w * h, shape=(h, w, 3), strides=(3 * w - 3, 3, 1))
    for bad in (planar, overlap):
        with pytest.raises(ValueError, match="packed"):
            sff.sgm(bad, bad, FakeCuda(2 * w * h), FakeCuda(1 << 20))
    good = FakeCuda(3 * w * h, shape=(h, w, 3), strides=(3 * w, 3, 1))
    other = FakeCuda(3 * w * h, shape=(h, w - 1, 3), strides=(3 * w, 3, 1))
    with pytest.raises(ValueError, match="shape"):
        sff.sgm(good, other, FakeCuda(2 * w * h), FakeCuda(1 << 20))
