"""The C-ABI library builds, loads without a GPU, exports every function include/mfa.h
declares, and rejects bad arguments on the host before touching CUDA (CPU only)."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(mfa_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libmfa():
    from paper_2312_15073_gb300 import build
    build.build()
    import paper_2312_15073_gb300 as mfa
    return mfa.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("mfa_model_create", "mfa_decode", "mfa_render", "mfa_model_destroy", "mfa_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(libmfa):
    from paper_2312_15073_gb300 import LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in exported, name
        assert hasattr(libmfa, name)


def test_host_side_argument_checks(libmfa):
    import paper_2312_15073_gb300 as mfa
    L = libmfa
    assert L.mfa_decode(None, None, 10, None, None) == -1
    assert "NULL" in L.mfa_last_error().decode()
    assert L.mfa_decode(None, None, 0, None, None) == -1          # model is still required
    assert L.mfa_locate_spans(None, None, -1, None) == -1
    cam = mfa.camera(dict(projection=0, eye=(0, 0, 2), target=(0, 0, 0), up=(0, 1, 0), ortho_height=1.0))
    tf = mfa.transfer_fn(np.zeros((4, 4)))
    assert L.mfa_render(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None) == -1
    # host-buffer forms check the same way, before any device work
    assert L.mfa_decode_host(None, None, 10, None, None) == -1
    assert L.mfa_decode_host(None, None, -3, None, None) == -1
    assert L.mfa_render_host(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, None) == -1
    assert "NULL" in L.mfa_last_error().decode()
    assert L.mfa_render_segments(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, None, None) == -1
    assert "blocks" in L.mfa_last_error().decode()
    g = (ctypes.c_int * 3)(2, 0, 1)
    assert L.mfa_render_segments(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, g, None, None) == -1
    g = (ctypes.c_int * 3)(8, 8, 2)
    assert L.mfa_render_segments(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, g, None, None) == -1
    assert "at most 64" in L.mfa_last_error().decode()
    assert L.mfa_render_iso(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, ctypes.c_float(float("nan")),
                            None, None, None) == -1
    assert "finite" in L.mfa_last_error().decode()
    assert L.mfa_render_iso(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, ctypes.c_float(0.5),
                            None, None, None) == -1
    # the ground-truth render and the image metrics check their arguments first too
    assert L.mfa_render_ml(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, None) == -1
    assert "signal" in L.mfa_last_error().decode()
    sig = mfa._MlSignal(6.0, -0.25)
    assert L.mfa_render_ml(ctypes.byref(sig), ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, None) == -1
    assert "alpha" in L.mfa_last_error().decode()
    sig = mfa._MlSignal(6.0, 0.25)
    assert L.mfa_render_ml(ctypes.byref(sig), ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, None) == -1
    assert "NULL" in L.mfa_last_error().decode()
    q = mfa._Quality()
    assert L.mfa_image_compare(None, None, 16, 16, ctypes.byref(q)) == -1
    assert L.mfa_image_compare(0x1004, 0x2000, 16, 16, ctypes.byref(q)) == -1
    assert "aligned" in L.mfa_last_error().decode()
    assert L.mfa_image_compare(0x1000, 0x2000, 10, 16, ctypes.byref(q)) == -1
    assert "11..32768" in L.mfa_last_error().decode()
    # render options are checked before anything else: variants 0..8, tile shapes 0..3
    opts = mfa._Opts()
    opts.variant = 9
    assert L.mfa_render_ex(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, ctypes.byref(opts)) == -1
    assert "0..8" in L.mfa_last_error().decode()
    opts.variant, opts.tile_shape = 7, 4
    assert L.mfa_render_ex(None, ctypes.byref(cam), ctypes.byref(tf.struct), 8, 8, 8, None, ctypes.byref(opts)) == -1
    assert "tile_shape" in L.mfa_last_error().decode()
    # checkpoint calls check their arguments and the file before any device work
    assert L.mfa_model_get_ctrl(None, None) == -1
    assert L.mfa_model_save(None, b"/nonexistent/x.mfa") == -1
    assert not L.mfa_model_load(b"/nonexistent/x.mfa")
    assert "cannot open" in L.mfa_last_error().decode()
    import tempfile, os, struct
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "bad.mfa")
        open(p, "wb").write(b"NOTMFA!!" + bytes(56))
        assert not L.mfa_model_load(p.encode())
        assert "not an MFA model file" in L.mfa_last_error().decode()
        hdr = b"MFAMODL1" + struct.pack("<i3i3ii6i", 1, 3, 3, 9, 8, 8, 8, 1, *([0] * 6))
        open(p, "wb").write(hdr)
        assert not L.mfa_model_load(p.encode())
        assert "degree" in L.mfa_last_error().decode()
        hdr = b"MFAMODL1" + struct.pack("<i3i3ii6i", 1, 3, 3, 3, 8, 8, 8, 1, *([0] * 6))
        open(p, "wb").write(hdr + bytes(8 * 36))                 # knots but no control points
        assert not L.mfa_model_load(p.encode())
        assert "truncated" in L.mfa_last_error().decode()
    # model creation rejects bad degrees, counts and knots before any device work
    deg = (ctypes.c_int * 3)(3, 3, 5)
    nc = (ctypes.c_int * 3)(8, 8, 8)
    ctrl = np.zeros(512)
    assert not L.mfa_model_create(ctypes.byref(deg), ctypes.byref(nc), None, ctrl.ctypes.data, 0)
    assert "degree" in L.mfa_last_error().decode()
    deg = (ctypes.c_int * 3)(3, 3, 3)
    nc = (ctypes.c_int * 3)(8, 3, 8)
    assert not L.mfa_model_create(ctypes.byref(deg), ctypes.byref(nc), None, ctrl.ctypes.data, 0)
    assert "nctrl" in L.mfa_last_error().decode()
    nc = (ctypes.c_int * 3)(8, 8, 8)
    bad = np.array([0, 0, 0, 0, 0.5, 0.4, 0.8, 0.9, 1, 1, 1, 1.0])      # decreasing
    ok = np.array([0, 0, 0, 0, 0.2, 0.4, 0.8, 0.9, 1, 1, 1, 1.0])
    kp = (ctypes.c_void_p * 3)(ok.ctypes.data, bad.ctypes.data, None)
    assert not L.mfa_model_create(ctypes.byref(deg), ctypes.byref(nc), ctypes.byref(kp), ctrl.ctypes.data, 0)
    assert "knots[1]" in L.mfa_last_error().decode()
    unclamped = np.array([0, 0, 0, 0.1, 0.2, 0.4, 0.8, 0.9, 1, 1, 1, 1.0])
    kp = (ctypes.c_void_p * 3)(unclamped.ctypes.data, None, None)
    assert not L.mfa_model_create(ctypes.byref(deg), ctypes.byref(nc), ctypes.byref(kp), ctrl.ctypes.data, 0)
    assert "knots[0]" in L.mfa_last_error().decode()
    assert not L.mfa_model_create_ex(ctypes.byref(deg), ctypes.byref(nc), None, ctrl.ctypes.data, 0, 0)
    assert "storage" in L.mfa_last_error().decode()
    L.mfa_model_create_opts.restype = ctypes.c_void_p
    for window in (-1, 4, 7):                                           # not an MFA_WINDOW_* choice
        assert not L.mfa_model_create_opts(ctypes.byref(deg), ctypes.byref(nc), None, ctrl.ctypes.data, 0, 1, window)
        assert "window" in L.mfa_last_error().decode()
    # per-cell patches (MFA_WINDOW_PATCH = 3): degree 3 on every axis
    deg2 = (ctypes.c_int * 3)(3, 2, 3)
    assert not L.mfa_model_create_opts(ctypes.byref(deg2), ctypes.byref(nc), None, ctrl.ctypes.data, 0, 1, 3)
    assert "MFA_WINDOW_PATCH" in L.mfa_last_error().decode()
    L.mfa_model_destroy(None)          # a no-op


def test_library_fails_loudly_when_missing(monkeypatch, tmp_path):
    import paper_2312_15073_gb300 as mfa
    monkeypatch.setattr(mfa, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(mfa, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        mfa.lib()


def test_tune_cache_file_errors(libmfa, tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("# header only\nnot a line\n")
    assert libmfa.mfa_tune_load(str(bad).encode()) == -1
    assert libmfa.mfa_tune_load(str(tmp_path / "missing.txt").encode()) == -1
    ok = tmp_path / "ok.txt"
    ok.write_text("4 1 10 10 1 7 2 3 1.5\n4 1 10 10 1 7 9 3 1.5\n")      # second line: bad variant, skipped
    assert libmfa.mfa_tune_load(str(ok).encode()) == 0
    out = tmp_path / "out.txt"
    assert libmfa.mfa_tune_save(str(out).encode()) == 0
    assert "4 1 10 10 1 7 2 3" in out.read_text()


def test_tune_cache_from_the_environment(libmfa, tmp_path):
    """MFA_TUNE_CACHE: the named file's choices are read on the first use of the cache (a
    fresh process; no GPU needed to read and write the cache)."""
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    cache.write_text("# q storage pixel_bucket sample_bucket uniform size_bucket variant tile_shape ms\n"
                     "3 2 9 9 0 8 7 1 2.5\n")
    out = tmp_path / "out.txt"
    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); "
            "sys.exit(L.mfa_tune_save(sys.argv[2].encode()))")
    env = dict(os.environ, MFA_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code, libmfa._name, str(out)], env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "3 2 9 9 0 8 7 1" in out.read_text()
    env["MFA_TUNE_CACHE"] = str(tmp_path / "missing.txt")          # a missing file is an empty cache
    r = subprocess.run([sys.executable, "-c", code, libmfa._name, str(out)], env=env, capture_output=True, text=True)
    assert r.returncode == 0 and "3 2 9 9" not in out.read_text()
