"""Checkpoint / resume: a run interrupted and resumed from its checkpoint is
bit-identical to the uninterrupted run; a checkpoint loads into either
storage precision; malformed files are rejected."""
import numpy as np
import pytest

from workloads import FP32_COMPRESSED, FP64_PLAIN, HOT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1310_7087_gb300 import build
    build.build()
    import paper_1310_7087_gb300 as q
    return q


@pytest.mark.parametrize("group,precision", [(3, FP32_COMPRESSED), (2, FP64_PLAIN), (3, FP64_PLAIN)])
def test_resume_is_bit_identical(q, tmp_path, group, precision):
    path = str(tmp_path / "state.qcd")
    a = q.Lattice(group, 4, 4, 5.7 if group == 3 else 2.3, 1, precision, HOT, 21, nhit=3)
    a.sweep(2, 2, 21)
    a.save(path)
    b = q.Lattice.load(path, precision)
    assert b.sweep_counter == a.sweep_counter == 2
    assert np.array_equal(a.get_links(), b.get_links())
    a.sweep(2, 2, 21)
    b.sweep(2, 2, 21)
    assert np.array_equal(a.get_links(), b.get_links())
    assert a.measure() == b.measure()
    assert a.exhausted == b.exhausted
    a.close()
    b.close()


def test_checkpoint_is_portable_across_storage(q, tmp_path):
    path = str(tmp_path / "fp64.qcd")
    a = q.Lattice(3, 4, 2, 6.0, 2, FP64_PLAIN, HOT, 3)
    a.sweep(1, 1, 3)
    a.save(path)
    b = q.Lattice.load(path, FP32_COMPRESSED)
    ref, got = a.get_links(), b.get_links()
    # FP32 keeps rows 1-2 rounded to FP32 and rebuilds row 3
    assert np.abs(got - ref).max() < 5e-7
    assert abs(b.measure()[0][0] - a.measure()[0][0]) < 1e-6
    a.close()
    b.close()


def test_malformed_checkpoint_is_rejected(q, tmp_path):
    bad = tmp_path / "bad.qcd"
    bad.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(q.QcdError) as e:
        q.qcd_lattice_load(str(bad))
    assert e.value.code == q.QCD_ERR_INVALID_ARG
    a = q.Lattice(2, 4, 2, 2.0, 0, FP32_COMPRESSED, HOT, 1)
    path = tmp_path / "cut.qcd"
    a.save(str(path))
    data = path.read_bytes()
    path.write_bytes(data[: len(data) // 2])
    with pytest.raises(q.QcdError):
        q.qcd_lattice_load(str(path))
    with pytest.raises(q.QcdError):
        q.qcd_lattice_load(str(tmp_path / "missing.qcd"))
    a.close()
