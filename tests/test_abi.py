"""Host-side checks that need no GPU: the C-ABI library builds, loads, and exports every
entry point include/rbws.h declares; the product package never touches the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"RBWS_API[^;{]*?\b(rbws_\w+)\s*\(", text, flags=re.S))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2311_13862_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for must in ("rbws_problem_create", "rbws_problem_destroy", "rbws_apply_operator",
                 "rbws_offline_greedy", "rbws_solve_batch", "rbws_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rbws_\w+)\b", out))
    assert set(declared_symbols()) <= exported


def test_errors_without_gpu_are_reported_not_hidden(lib_path):
    from paper_2311_13862_gb300 import rbws
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(rbws.RbwsError):
        rbws.rbws_problem_create((8, 8, 8), (2, 1, 1))


def test_invalid_arguments_are_rejected(lib_path):
    from paper_2311_13862_gb300 import rbws
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create((1, 8, 8), (2, 1, 1))
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create((8, 8, 8), (2, 1, 1), Q=3)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_13862_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, flags=re.M), f
                assert "rbws_oracle" not in text and "liborc" not in text, f


def test_options_default_sets_every_field(lib_path):
    """rbws_options_default must overwrite every field (internal callers rely on it)."""
    import ctypes as C
    from paper_2311_13862_gb300 import rbws
    o = rbws.rbws_options()
    C.memset(C.byref(o), 0xAB, C.sizeof(o))
    rbws._lib().rbws_options_default(C.byref(o))
    assert o.max_iters == 20000 and o.precond == rbws.PREC_JACOBI and o.precision == rbws.FP64
    assert o.max_restarts == 3 and o.inner_tol == 0.0 and o.max_outer == 10 and o.check_every == 0
    assert o.stream is None and not o.profile and o.relres_hist is None and o.hist_len == 0
    assert o.wait_cycles == 0 and o.ru_mode == 0 and o.persistent == 0


def _ckpt_bytes(nx=4, ny=3, nz=2, blocks=(2, 1, 1), N=2, checksum_ok=True, submap=None, Q=None, faces=None):
    """A checkpoint in the library's documented layout (no network, f = 1; the subdomain map
    submap [n] uint8 with Q subdomains if given, else the block rule; with faces = (kfx, kfy,
    kfz), a face-field problem of Q terms: version 4, the axes and the face arrays first)."""
    import struct
    import numpy as np
    n = nx * ny * nz
    Q = blocks[0] * blocks[1] * blocks[2] if submap is None and faces is None else Q
    version, has_map, head = 2, int(submap is not None), b""
    if faces is not None:
        version, has_map = 4, 2
        # rbws_axes: kappa_scale f64[3], neumann_hi i32[3], reserved i32
        head = struct.pack("<3d4i", 1.0, 1.0, 1.0, 0, 0, 0, 0)
        head += b"".join(np.ascontiguousarray(a, dtype=np.float64).tobytes() for a in faces)
    payload = (head + (b"" if submap is None else np.asarray(submap, dtype=np.uint8).tobytes())
               + np.arange(N * n, dtype=np.float64).tobytes() + np.ones(Q * N * N).tobytes()
               + np.ones(N).tobytes())
    # i32 fields: nx ny nz bx by bz Q has_f N net_H net_N has_map, then 4 bytes of padding
    hdr = struct.pack("<8sI12i4x2dQ", b"RBWSPRB1", version, nx, ny, nz, blocks[0], blocks[1], blocks[2], Q, 0, N,
                      0, 0, has_map, 0.0, 0.0, len(payload))
    h = 1469598103934665603
    for c in payload:
        h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    if not checksum_ok:
        h ^= 1
    return hdr + payload + struct.pack("<Q", h)


def test_checkpoint_loader_rejects_bad_files(tmp_path, lib_path):
    from paper_2311_13862_gb300 import rbws
    bad = tmp_path / "garbage.bin"
    bad.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(rbws.RbwsError, match="not a checkpoint"):
        rbws.rbws_load(bad)
    good = _ckpt_bytes()
    trunc = tmp_path / "trunc.bin"
    trunc.write_bytes(good[:-20])
    with pytest.raises(rbws.RbwsError, match="truncated"):
        rbws.rbws_load(trunc)
    wrong = tmp_path / "wrong.bin"
    wrong.write_bytes(_ckpt_bytes(checksum_ok=False))
    with pytest.raises(rbws.RbwsError, match="checksum"):
        rbws.rbws_load(wrong)


def test_checkpoint_loader_accepts_a_valid_file_up_to_device_set_up(tmp_path, lib_path):
    import torch
    from paper_2311_13862_gb300 import rbws
    if torch.cuda.is_available():
        pytest.skip("GPU present: covered by the GPU checkpoint test")
    ok = tmp_path / "ok.bin"
    ok.write_bytes(_ckpt_bytes())
    with pytest.raises(rbws.RbwsError, match="CUDA"):  # parsed and verified; no device here
        rbws.rbws_load(ok)
    # with an explicit map: the map travels in the payload and reaches device set-up
    ok.write_bytes(_ckpt_bytes(submap=[0, 1, 1, 0] + [0] * 20, Q=2))
    with pytest.raises(rbws.RbwsError, match="CUDA"):
        rbws.rbws_load(ok)
    ok.write_bytes(_ckpt_bytes(submap=[0, 2, 1, 0] + [0] * 20, Q=2))
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):  # map value 2 >= Q
        rbws.rbws_load(ok)
    # a face-field problem (version 4): the face arrays travel in the payload
    import numpy as np
    nx, ny, nz, Q = 4, 3, 2, 2
    kfx, kfy, kfz = np.ones((Q, nz, ny, nx + 1)), np.ones((Q, nz, ny + 1, nx)), np.ones((Q, nz + 1, ny, nx))
    ok.write_bytes(_ckpt_bytes(Q=Q, faces=(kfx, kfy, kfz)))
    with pytest.raises(rbws.RbwsError, match="CUDA"):
        rbws.rbws_load(ok)
    kfx[:, 0, 0, 0:2], kfy[:, 0, 0:2, 0], kfz[:, 0:2, 0, 0] = 0.0, 0.0, 0.0  # node (0, 0, 0): no face left
    ok.write_bytes(_ckpt_bytes(Q=Q, faces=(kfx, kfy, kfz)))
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_load(ok)
    ok.write_bytes(_ckpt_bytes(Q=Q, faces=(kfx, kfy, kfz))[:-9])
    with pytest.raises(rbws.RbwsError, match="truncated"):
        rbws.rbws_load(ok)


def test_explicit_maps_are_checked_before_the_device(lib_path):
    """Explicit maps are cut into boxes by their interface planes; the limits (segments per
    axis, coefficient classes) and value checks run on the host, visible without a GPU."""
    import numpy as np
    import torch
    from paper_2311_13862_gb300 import rbws
    grid = (6, 5, 4)
    m = np.zeros((4, 5, 6), dtype=np.uint8)
    m[:, :, 2:] = 1
    m[1:3, 1:3, 2:4] = 2                 # an inclusion: boxes between the cut planes
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create(grid, None, Q=2, subdomain_map=m)  # value 2 >= Q
    many = np.zeros((4, 5, 70), dtype=np.uint8)
    many[:, :, ::2] = 1                  # 70 segments along x: more than the limit
    with pytest.raises(rbws.RbwsError, match="UNSUPPORTED.*segments"):
        rbws.rbws_problem_create((70, 5, 4), None, Q=2, subdomain_map=many)
    i = np.arange(60) // 2 % 2           # 30 segments of 2 nodes per axis: 60^3 classes
    cb = (i[:, None, None] ^ i[None, :, None] ^ i[None, None, :]).astype(np.uint8)
    with pytest.raises(rbws.RbwsError, match="UNSUPPORTED.*classes"):
        rbws.rbws_problem_create((60, 60, 60), None, Q=2, subdomain_map=cb)
    if not torch.cuda.is_available():
        with pytest.raises(rbws.RbwsError, match="CUDA"):  # accepted; no device here
            rbws.rbws_problem_create(grid, None, Q=3, subdomain_map=m)


def test_face_fields_are_checked_before_the_device(lib_path):
    """Face-field problems: sizes, face values and rows that are zero in every term are
    rejected on the host; a valid field reaches device set-up."""
    import numpy as np
    import torch
    from paper_2311_13862_gb300 import rbws
    nx, ny, nz, Q = 5, 4, 3, 2
    kfx = np.ones((Q, nz, ny, nx + 1))
    kfy = np.ones((Q, nz, ny + 1, nx))
    kfz = np.ones((Q, nz + 1, ny, nx))
    with pytest.raises(rbws.RbwsError, match="INVALID_ARG"):
        rbws.rbws_problem_create_field((1, ny, nz), kfx[:, :, :, :2], kfy[:, :, :, :1], kfz[:, :, :, :1])
    for arr, val in ((kfx, -1.0), (kfy, np.nan), (kfz, np.inf)):
        bad = arr.copy()
        bad[1, 1, 1, 1] = val
        args = [kfx, kfy, kfz]
        args[[id(a) for a in (kfx, kfy, kfz)].index(id(arr))] = bad
        with pytest.raises(rbws.RbwsError, match="finite and >= 0"):
            rbws.rbws_problem_create_field((nx, ny, nz), *args)
    # node (2, 1, 1): its six faces zero in both terms
    zx, zy, zz = kfx.copy(), kfy.copy(), kfz.copy()
    zx[:, 1, 1, 2:4] = 0.0
    zy[:, 1, 1:3, 2] = 0.0
    zz[:, 1:3, 1, 2] = 0.0
    with pytest.raises(rbws.RbwsError, match=r"node \(2, 1, 1\) has no positive face"):
        rbws.rbws_problem_create_field((nx, ny, nz), zx, zy, zz)
    # zero in one term only: the other term keeps the row
    zx[1], zy[1], zz[1] = kfx[1], kfy[1], kfz[1]
    if not torch.cuda.is_available():
        with pytest.raises(rbws.RbwsError, match="CUDA"):  # accepted; no device here
            rbws.rbws_problem_create_field((nx, ny, nz), zx, zy, zz)
