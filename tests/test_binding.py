"""Host logic of the Python binding (CPU): no CPU fallback, and the stream
ordering of the tensors the wrapper makes."""
import contextlib

import pytest

from paper_1603_08328_gb300 import lem


def test_no_cpu_path():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU path"):
        lem.Stereo(None, None)
    with pytest.raises(RuntimeError, match="no CPU path"):
        lem.ProposalNet()


class _FakeCuda:
    def __init__(self):
        self.current = "default"

    @contextlib.contextmanager
    def stream(self, s):
        prev, self.current = self.current, s
        try:
            yield
        finally:
            self.current = prev


class _FakeTorch:
    def __init__(self):
        self.cuda = _FakeCuda()


class _Obj:
    def __init__(self, stream):
        self.torch = _FakeTorch()
        self.stream = stream

    @lem._on_own_stream
    def work(self, x, y=0):
        return self.torch.cuda.current, x + y

    @lem._on_own_stream
    def fails(self):
        raise ValueError("inside")


def test_methods_run_on_the_objects_stream():
    o = _Obj("side")
    assert o.work(1, y=2) == ("side", 3)
    assert o.torch.cuda.current == "default"
    with pytest.raises(ValueError):
        o.fails()
    assert o.torch.cuda.current == "default"


def test_tensor_methods_are_stream_ordered():
    """Every wrapper method that allocates or copies tensors runs with the handle's
    stream current."""
    for cls, names in [(lem.Stereo, ["unary", "pairwise", "mincut", "labels", "set_labels", "planes",
                                     "proposals_of", "postprocess", "set_proposals", "proposals",
                                     "cnn_features", "cnn_targets"]),
                       (lem.ProposalNet, ["forward", "gradients", "train_step"])]:
        for n in names:
            assert getattr(getattr(cls, n), "__wrapped__", None) is not None, f"{cls.__name__}.{n}"
