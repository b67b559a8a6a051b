"""The batched autotuner's driver (no GPU): the first call measures and caches,
later calls restore from the cache, `force` measures again, a damaged cache is
treated as empty, and keys separate GPUs and reservations."""
from paper_1710_10989_gb300 import tuner


class FakeHandle:
    device = 0

    def __init__(self, result=(0xF0F0, 152), shapes=(0x3, 0xC, 0x1)):
        self.result = result
        self.shapes = shapes
        self.tuned = 0
        self.installed = None
        self.installed_shapes = "unset"

    def batch_tune(self, max_n, tol):
        self.tuned += 1
        return self.result

    def batch_get_shapes(self):
        return self.shapes

    def batch_set_tuning(self, mask, ctas):
        self.installed = (mask, ctas)

    def batch_set_shapes(self, masks):
        self.installed_shapes = masks


def test_measure_then_restore(tmp_path):
    path = str(tmp_path / "t.json")
    h = FakeHandle()
    assert tuner.tuned(h, 256, path=path, gpu="G") == (0xF0F0, 152)
    assert h.tuned == 1 and h.installed is None      # measured: bbc_batch_tune installed it itself
    h2 = FakeHandle(result=(1, 1))
    assert tuner.tuned(h2, 256, path=path, gpu="G") == (0xF0F0, 152)
    assert h2.tuned == 0 and h2.installed == (0xF0F0, 152)
    assert list(h2.installed_shapes) == [0x3, 0xC, 0x1]   # the tuned product shapes come back too
    assert tuner.tuned(h2, 256, path=path, gpu="G", force=True) == (1, 1)
    assert h2.tuned == 1


def test_keys_separate_gpus_and_reservations(tmp_path):
    path = str(tmp_path / "t.json")
    tuner.tuned(FakeHandle((1, 10)), 256, path=path, gpu="A")
    tuner.tuned(FakeHandle((2, 20)), 128, path=path, gpu="A")
    tuner.tuned(FakeHandle((3, 30)), 256, path=path, gpu="B")
    data = tuner.load(path)
    assert len(data) == 3
    h = FakeHandle((9, 9))
    assert tuner.tuned(h, 128, path=path, gpu="A") == (2, 20) and h.tuned == 0


def test_damaged_cache_is_ignored(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    h = FakeHandle()
    assert tuner.tuned(h, 64, path=str(path), gpu="G") == (0xF0F0, 152)
    assert h.tuned == 1


def test_entry_without_shapes_restores_default_shapes(tmp_path):
    path = str(tmp_path / "t.json")
    tuner.save(path, {tuner.cache_key("G", 256, 0.0): {"split_mask": 5, "ctas": 7}})
    h = FakeHandle()
    assert tuner.tuned(h, 256, path=path, gpu="G") == (5, 7)
    assert h.installed_shapes is None
