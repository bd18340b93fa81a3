"""The on-disk cache of batched-launch tunings (host logic, no GPU): a
batch's key changes with the GPU model and with any property of any
problem, entries round-trip, and a missing, corrupt or mismatched file
reads as a miss rather than an error."""
import json

import numpy as np

import synth
from paper_1609_00958_gb300 import tuning_cache as tc


def _sig(cg, dtype="float32", shape=(32, 32, 32), h=(1.0, 1.0, 1.0), origin=None, weight="lin", fov=0.0):
    d = tc.geometry_digest(cg.src, cg.det_origin, cg.det_u, cg.det_v, cg.nu, cg.nv)
    return tc.problem_signature(dtype, shape, h, origin, d, weight, fov)


def test_key_depends_on_gpu_and_every_problem_property():
    cg = synth.circular(8, 16, 12, 100.0, 200.0, 1.5)
    base = [_sig(cg), _sig(cg, dtype="bfloat16")]
    k = tc.batch_key("NVIDIA GB300", base)
    assert k == tc.batch_key("NVIDIA GB300", [_sig(cg), _sig(cg, dtype="bfloat16")])
    assert k != tc.batch_key("NVIDIA B200", base)
    assert k != tc.batch_key("NVIDIA GB300", base[::-1])
    moved = synth.circular(8, 16, 12, 100.0, 200.0, 1.5)
    moved.src[3, 0] += 1e-9
    variants = [[_sig(moved), base[1]], [_sig(cg, shape=(32, 32, 33)), base[1]],
                [_sig(cg, h=(1.0, 1.0, 1.1)), base[1]], [_sig(cg, origin=(0.0, 0.0, 0.0)), base[1]],
                [_sig(cg, weight="spl"), base[1]], [_sig(cg, fov=10.0), base[1]],
                [_sig(synth.circular(8, 16, 13, 100.0, 200.0, 1.5)), base[1]]]
    keys = {tc.batch_key("NVIDIA GB300", v) for v in variants}
    assert len(keys) == len(variants) and k not in keys


def test_store_and_lookup_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tunings.json")
    assert tc.lookup(path, "k1", 2) is None                       # no file yet
    tc.store(path, "k1", "GPU", [(4, 16), (1, 8)])
    tc.store(path, "k2", "GPU", [(2, 4)])
    assert tc.lookup(path, "k1", 2) == [(4, 16), (1, 8)]
    assert tc.lookup(path, "k2", 1) == [(2, 4)]
    assert tc.lookup(path, "k1", 3) is None                       # another problem count
    tc.store(path, "k1", "GPU", [(2, 1), (4, 64)])                  # replaced
    assert tc.lookup(path, "k1", 2) == [(2, 1), (4, 64)]
    assert json.load(open(path))["k2"]["gpu"] == "GPU"


def test_bad_files_and_entries_are_misses(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    assert tc.lookup(str(path), "k", 1) is None
    path.write_text(json.dumps({"k": {"tunings": [[3, 16]]}}))      # tile_u 3 is not a shape
    assert tc.lookup(str(path), "k", 1) is None
    path.write_text(json.dumps({"k": {"tunings": [[4, 0]]}}))
    assert tc.lookup(str(path), "k", 1) is None
    path.write_text(json.dumps([1, 2]))
    assert tc.lookup(str(path), "k", 1) is None
    tc.store(str(path), "k", "GPU", [(4, 8)])                        # a bad file is replaced
    assert tc.lookup(str(path), "k", 1) == [(4, 8)]


def test_geometry_digest_sees_the_detector_size():
    cg = synth.circular(3, 16, 12, 100.0, 200.0, 1.5)
    a = tc.geometry_digest(cg.src, cg.det_origin, cg.det_u, cg.det_v, 16, 12)
    b = tc.geometry_digest(cg.src, cg.det_origin, cg.det_u, cg.det_v, 12, 16)
    assert a != b
    # the arrays are taken as float64 whatever their input type
    assert a == tc.geometry_digest(cg.src.tolist(), cg.det_origin, cg.det_u, cg.det_v, 16, 12)
