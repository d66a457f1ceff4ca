"""The C-ABI library loads on a machine without a GPU, exports every entry point
declared in include/lbm_sc.h, and its host-only calls validate arguments."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_sc_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 12
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(so, name), name
    assert declared == set(lib.EXPORTS) | (declared - set(lib.EXPORTS))
    assert set(lib.EXPORTS) <= declared


def test_workspace_sizes(lib):
    p = lib.make_params(lib.LBM_D3Q19, (10, 12, 14), 1.0, 1.0, 2.0, "f32")
    n = 10 * 12 * 14
    ws = lib.lbm_sc_workspace_bytes(p)
    assert ws >= 2 * 2 * 19 * n * 4
    p32 = lib.make_params(lib.LBM_D3Q19, (10, 12, 200), 1.0, 1.0, 2.0, "f32")
    p16 = lib.make_params(lib.LBM_D3Q19, (10, 12, 200), 1.0, 1.0, 2.0, "bf16")
    assert lib.lbm_sc_workspace_bytes(p16) < 0.7 * lib.lbm_sc_workspace_bytes(p32)
    # ghost-padded planes: pitch multiple of 16 bytes, one-node images on every side
    for prec, eb in (("f64", 8), ("f32", 4), ("bf16", 2)):
        pp = lib.make_params(lib.LBM_D3Q19, (10, 12, 14), 1.0, 1.0, 2.0, prec)
        h = lib.lbm_sc_create(pp, 256 * 1024, lib.lbm_sc_workspace_bytes(pp), 0)
        e, q, px, py, gx, gy, _ = lib.lbm_sc_layout(h)
        lib.lbm_sc_destroy(h)
        assert e == eb and q == 19 and gx * eb == 128 and gy == 2
        assert (px * eb) % 128 == 0 and px >= 14 + gx + 16 // eb and py == 12 + 4
        assert lib.lbm_sc_workspace_bytes(pp) >= 2 * 2 * 19 * px * py * 10 * eb
    p64 = lib.make_params(lib.LBM_D2Q9, (12, 14), 1.0, 1.0, 2.0, "f64")
    assert lib.lbm_sc_workspace_bytes(p64) >= 2 * 2 * 9 * 12 * 14 * 8
    assert lib.lbm_sc_host_staging_bytes(p) >= 6 * n * 4


@pytest.mark.parametrize("bad", [
    dict(tau_A=0.5), dict(tau_B=0.3), dict(nx=0), dict(ny=-1), dict(nz=0), dict(lattice=7), dict(precision=9),
])
def test_invalid_params_rejected(lib, bad):
    p = lib.make_params(lib.LBM_D3Q19, (4, 4, 4), 1.0, 1.0, 2.0, "f32")
    for k, v in bad.items():
        setattr(p, k, v)
    assert lib.lbm_sc_workspace_bytes(p) == 0
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_sc_create(p, 1 << 20, 1 << 30, 0)
    assert e.value.status == lib.LBM_ERR_INVALID_ARG


def test_d2q9_requires_nz_1_and_size_limit(lib):
    p = lib.make_params(lib.LBM_D2Q9, (4, 4), 1.0, 1.0, 2.0, "f32")
    p.nz = 2
    assert lib.lbm_sc_workspace_bytes(p) == 0
    big = lib.make_params(lib.LBM_D3Q19, (2048, 1024, 1024), 1.0, 1.0, 2.0, "f32")
    assert lib.lbm_sc_workspace_bytes(big) == 0  # N >= 2^31


def test_create_checks_workspace_without_touching_the_gpu(lib):
    p = lib.make_params(lib.LBM_D2Q9, (8, 8), 1.0, 1.0, 2.0, "f32")
    need = lib.lbm_sc_workspace_bytes(p)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_sc_create(p, 256 * 1024, need - 1, 0)
    assert e.value.status == lib.LBM_ERR_OUT_OF_MEMORY
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_sc_create(p, 256 * 1024 + 8, need, 0)  # misaligned
    assert e.value.status == lib.LBM_ERR_INVALID_ARG
    h = lib.lbm_sc_create(p, 256 * 1024, need, 0)  # a fake address: create does not dereference it
    eb, q, px, py, gx, gy, ptr = lib.lbm_sc_layout(h)
    assert (eb, q, ptr) == (4, 9, 256 * 1024)
    assert gx == 32 and gy == 2 and py == 8 + 2 * gy and px >= 8 + gx + 4 and (px * eb) % 128 == 0
    with pytest.raises(lib.LbmError):
        lib.lbm_sc_step(h, -1)
    lib.lbm_sc_destroy(h)


def test_tuning_validation(lib):
    p = lib.make_params(lib.LBM_D3Q19, (40, 8, 64), 1.0, 1.0, 2.0, "f32")
    h = lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0)
    try:
        for t in range(len(lib.TILES)):
            tx, ty = lib.TILES[t]
            cx, cy = lib.TILE_CLUSTER[t]
            # TMA tiles: at least one tile in x and y, tile counts (ragged tiles included) divisible by the cluster
            fits = lib.TILE_KIND[t] != 5 or (64 >= tx and 8 >= ty and -(-64 // tx) % cx == 0 and -(-8 // ty) % cy == 0)
            fits = fits and lib.TILE_KIND[t] != 6  # 16-bit storage only
            fits = fits and lib.TILE_KIND[t] != lib.RETIRED  # removed kernels: every call is rejected
            if not fits:
                with pytest.raises(lib.LbmError):
                    lib.lbm_sc_set_tuning(h, t, 0)
                continue
            lib.lbm_sc_set_tuning(h, t, 0)
            assert lib.lbm_sc_get_tuning(h)[0] == t
        lib.lbm_sc_set_tuning(h, 1, 500)
        assert lib.lbm_sc_get_tuning(h) == (1, 40)  # clamped to nz
        for bad in ((-1, 0), (len(lib.TILES), 0), (0, -3)):
            with pytest.raises(lib.LbmError):
                lib.lbm_sc_set_tuning(h, *bad)
    finally:
        lib.lbm_sc_destroy(h)
    # the three-plane register kernels exist for D3Q19 with 32-bit or reference-offset storage, the
    # TMA kernels for D3Q19 (rest-offset storage runs only the kernels that pull through the generic
    # node loads and the 16-bit TMA kernel); retired ids are rejected everywhere
    for lat, shape, prec in ((lib.LBM_D2Q9, (8, 8), "f32"), (lib.LBM_D3Q19, (8, 8, 8), "f64"),
                             (lib.LBM_D3Q19, (8, 8, 8), "bf16"), (lib.LBM_D3Q19, (8, 8, 8), "bf16_rest"),
                             (lib.LBM_D2Q9, (8, 8), "f16_rest")):
        p = lib.make_params(lat, shape, 1.0, 1.0, 2.0, prec)
        h = lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0)
        try:
            for t in range(len(lib.TILES)):
                ok = lib.tile_supported(t, lat, p.precision)
                kind = lib.TILE_KIND[t]
                assert ok == (kind in (0, 3)
                              or (kind == 4 and lat == lib.LBM_D3Q19 and prec in ("f32", "bf16", "f16"))
                              or (kind == 6 and lat == lib.LBM_D3Q19 and prec in ("bf16", "bf16_rest")))
                if kind in (5, 6):  # TMA kernels also need one full tile in x and y
                    ok = False
                if ok:
                    lib.lbm_sc_set_tuning(h, t, 0)
                else:
                    with pytest.raises(lib.LbmError):
                        lib.lbm_sc_set_tuning(h, t, 0)
        finally:
            lib.lbm_sc_destroy(h)


def test_rest_offset_storage_sizes(lib):
    """Rest-offset 16-bit storage: Q planes of 32-bit words (both species'
    16-bit offsets of a direction) plus one float2 density plane per buffer,
    about 84/152 of the FP32 bytes for D3Q19 (42/72 for D2Q9)."""
    for lat, shape, q in ((lib.LBM_D3Q19, (64, 64, 64), 19), (lib.LBM_D2Q9, (256, 256), 9),
                          (lib.LBM_D3Q19, (16, 64, 1024), 19)):
        ws, px = {}, {}
        for pr in ("f32", "bf16", "bf16_rest", "f16_rest"):
            p = lib.make_params(lat, shape, 1.0, 1.0, 2.0, pr)
            ws[pr] = lib.lbm_sc_workspace_bytes(p)
            h = lib.lbm_sc_create(p, 256 * 1024, ws[pr], 0)
            px[pr] = lib.lbm_sc_layout(h)[2]  # row pitch in values: 128-byte ghost margin, 128-byte rows
            lib.lbm_sc_destroy(h)
        assert ws["bf16_rest"] == ws["f16_rest"]
        ratio = (q * 4 + 8) * px["bf16_rest"] / ((2 * q * 4) * px["f32"])
        assert abs(ws["bf16_rest"] / ws["f32"] - ratio) < 0.01 * ratio, (lat, ws)
        assert ws["bf16_rest"] < ws["f32"]
        if shape[-1] >= 1024:  # wide rows: 16-bit offsets alone are the smallest (narrow rows differ in padding)
            assert ws["bf16"] < ws["bf16_rest"]
    assert ratio < 0.61  # wide rows: the padding is a small part
    p = lib.make_params(lib.LBM_D3Q19, (10, 12, 14), 1.0, 1.0, 2.0, "bf16_rest")
    h = lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0)
    try:
        eb, q, px, py, gx, gy, ptr = lib.lbm_sc_layout(h)
        assert (eb, q) == (4, 19)  # one 32-bit word holds both species of a direction
        assert gx * eb == 128 and (px * eb) % 128 == 0
        # both buffers hold the paired populations and the float2 density plane
        assert lib.lbm_sc_workspace_bytes(p) >= 2 * (19 * px * py * 10 * 4 + px * py * 10 * 8)
    finally:
        lib.lbm_sc_destroy(h)
    bad = lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.0, 6)
    assert lib.lbm_sc_workspace_bytes(bad) == 0


def test_status_strings(lib):
    for s in range(6):
        assert lib.lbm_sc_status_string(s).startswith("LBM_")
    assert "unknown" in lib.lbm_sc_status_string(99)


def test_host_alloc_argument_checks_without_touching_the_gpu(lib):
    """lbm_sc_host_alloc rejects a zero size or a NULL out pointer (and leaves *out
    NULL), lbm_sc_host_free of NULL is a no-op and of a zero size is rejected;
    none of these reaches a CUDA call."""
    so = lib.load()
    out = ctypes.c_void_p(1234)
    assert so.lbm_sc_host_alloc(ctypes.c_size_t(0), ctypes.byref(out)) == lib.LBM_ERR_INVALID_ARG
    assert out.value is None
    assert so.lbm_sc_host_alloc(ctypes.c_size_t(4096), None) == lib.LBM_ERR_INVALID_ARG
    assert so.lbm_sc_host_free(None, ctypes.c_size_t(4096)) == lib.LBM_OK
    assert so.lbm_sc_host_free(ctypes.c_void_p(4096), ctypes.c_size_t(0)) == lib.LBM_ERR_INVALID_ARG


def test_batch_workspace_and_validation(lib):
    """Batch sizing counts one descriptor per lattice and one 16-byte item per
    (x tile, y tile, z chunk); mixed lattice kinds or precisions, unknown tiles,
    odd graph chunks and short or misaligned workspaces are rejected before any
    device work."""
    shapes = [(40, 20, 24), (17, 33, 9), (64, 64, 64)]
    ps = [lib.make_params(lib.LBM_D3Q19, s, 1.0, 0.8, 2.0, "f32") for s in shapes]
    hs = [lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0) for p in ps]
    try:
        for tile, (tx, ty) in enumerate(lib.BATCH_TILES[:3]):
            for zc in (0, 8, 100):
                z = 32 if zc == 0 else zc
                items = sum(-(-nx // tx) * -(-ny // ty) * -(-nz // min(z, nz)) for nz, ny, nx in shapes)
                ws = lib.lbm_sc_batch_workspace_bytes(hs, tile, zc)
                assert ws >= items * 16 + len(hs) * 2 * 80
                assert ws < items * 16 + len(hs) * 2 * 200 + 1024
        assert lib.lbm_sc_batch_workspace_bytes(hs, len(lib.BATCH_TILES), 0) == 0
        for t in range(len(lib.BATCH_TILES)):
            tma = lib.BATCH_TILE_TMA[t]
            if t == lib.BATCH_TILE_REST:  # rest-offset storage only: no FP32 set fits
                assert all(lib.lbm_sc_batch_workspace_bytes(x, t, 0) == 0 for x in (hs, hs[1:], hs[2:]))
                continue
            # TMA-fed tiles need every lattice at least one tile wide (nx = 24 < 32 here)
            assert (lib.lbm_sc_batch_workspace_bytes(hs, t, 0) == 0) == tma
            assert lib.lbm_sc_batch_workspace_bytes(hs[2:], t, 0) > 0
            fits = not tma or lib.BATCH_TILES[t][0] <= 9
            assert (lib.lbm_sc_batch_workspace_bytes(hs[1:], t, 0) > 0) == fits  # nx = 9
        # the rest-offset TMA tile takes rest-offset lattices at least 32 x 8 (and nothing narrower)
        pr = [lib.make_params(lib.LBM_D3Q19, s, 1.0, 0.8, 2.0, prec) for s, prec in
              (((16, 8, 32), "bf16_rest"), ((16, 8, 24), "bf16_rest"), ((16, 8, 32), "f16_rest"))]
        hr = [lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0) for p in pr]
        try:
            assert lib.lbm_sc_batch_workspace_bytes(hr[:1], lib.BATCH_TILE_REST, 0) > 0
            assert lib.lbm_sc_batch_workspace_bytes(hr[2:], lib.BATCH_TILE_REST, 0) > 0
            assert lib.lbm_sc_batch_workspace_bytes(hr[:2], lib.BATCH_TILE_REST, 0) == 0  # 24 columns
            assert lib.lbm_sc_batch_workspace_bytes([hr[0], hr[2]], lib.BATCH_TILE_REST, 0) == 0  # two storages
            assert lib.lbm_sc_batch_workspace_bytes(hr[:1], 12, 0) == 0  # the FP32 TMA tiles take no 16-bit words
        finally:
            for h in hr:
                lib.lbm_sc_destroy(h)
        assert lib.lbm_sc_batch_workspace_bytes(hs, -1, 0) == 0
        assert lib.lbm_sc_batch_workspace_bytes(hs, 0, -1) == 0
        assert lib.lbm_sc_batch_workspace_bytes([], 0, 0) == 0
        p2 = lib.make_params(lib.LBM_D2Q9, (16, 16), 1.0, 1.0, 2.0, "f32")
        p16 = lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.0, "bf16")
        for other in (p2, p16):
            h2 = lib.lbm_sc_create(other, 256 * 1024, lib.lbm_sc_workspace_bytes(other), 0)
            try:
                assert lib.lbm_sc_batch_workspace_bytes(hs + [h2], 0, 0) == 0
                with pytest.raises(lib.LbmError):
                    lib.lbm_sc_batch_create(hs + [h2], 0, 0, 0, 256 * 1024, 1 << 30, 0)
            finally:
                lib.lbm_sc_destroy(h2)
        need = lib.lbm_sc_batch_workspace_bytes(hs, 0, 0)
        cases = [((0, 0, 3, 256 * 1024, need), lib.LBM_ERR_INVALID_ARG),    # odd graph chunk
                 ((0, 0, -2, 256 * 1024, need), lib.LBM_ERR_INVALID_ARG),
                 ((0, 0, 0, 256 * 1024 + 8, need), lib.LBM_ERR_INVALID_ARG),  # misaligned
                 ((0, 0, 0, 256 * 1024, need - 1), lib.LBM_ERR_OUT_OF_MEMORY),
                 ((9, 0, 0, 256 * 1024, need), lib.LBM_ERR_INVALID_ARG),
                 ((3, 0, 0, 256 * 1024, need), lib.LBM_ERR_INVALID_ARG),
                 ((6, 0, 0, 256 * 1024, need), lib.LBM_ERR_INVALID_ARG)]
        for args, status in cases:
            with pytest.raises(lib.LbmError) as e:
                lib.lbm_sc_batch_create(hs, *args, 0)
            assert e.value.status == status, args
        with pytest.raises(lib.LbmError):
            lib.lbm_sc_batch_step(0, 1)
        lib.lbm_sc_batch_destroy(0)  # a null batch is ignored
    finally:
        for h in hs:
            lib.lbm_sc_destroy(h)


def test_struct_layouts_match_the_header(lib, tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (gcc reads
    include/lbm_sc.h: sizes and the offset of every field)."""
    import subprocess
    structs = {"lbm_sc_params": lib.lbm_sc_params, "lbm_sc_diag": lib.lbm_sc_diag,
               "lbm_sc_window": lib.lbm_sc_window, "lbm_sc_tuning": lib.lbm_sc_tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm_sc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[name + "." + field]) == getattr(cls, field).offset, (name, field)


def test_body_force_must_be_finite(lib):
    for A in (float("nan"), float("inf")):
        p = lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.0, "f32", body_A=A)
        assert lib.lbm_sc_workspace_bytes(p) == 0
    p = lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.0, "f32", body_A=-1e-6)
    assert lib.lbm_sc_workspace_bytes(p) > 0


def test_forcing_scheme_rules(lib):
    """lbm_forcing: 0 and 1 only; Guo forcing on the register / low-register
    tiles and tile 34; the TMA batch tiles need the velocity shift."""
    assert lib.lbm_sc_workspace_bytes(lib.make_params(lib.LBM_D2Q9, (8, 8), 1.0, 1.0, 2.0, "f32", forcing=2)) == 0
    for lat, shape, prec in ((lib.LBM_D3Q19, (8, 8, 8), "f32"), (lib.LBM_D2Q9, (8, 8), "f64"),
                             (lib.LBM_D3Q19, (8, 8, 8), "bf16_rest")):
        p = lib.make_params(lat, shape, 1.0, 1.0, 2.0, prec, forcing="guo")
        assert lib.lbm_sc_workspace_bytes(p) > 0
        h = lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0)
        try:
            for t in range(len(lib.TILES)):
                kind = lib.TILE_KIND[t]
                ok = lib.tile_supported(t, lat, p.precision, lib.LBM_FORCING_GUO)
                assert ok == (kind in (0, 3) or (t == 34 and lat == lib.LBM_D3Q19 and prec == "f32"))
                if ok and kind in (0, 3):
                    lib.lbm_sc_set_tuning(h, t, 0)
                elif not ok:
                    with pytest.raises(lib.LbmError):
                        lib.lbm_sc_set_tuning(h, t, 0)
        finally:
            lib.lbm_sc_destroy(h)


def test_fe_model_rules(lib):
    """lbm_model: the FE model takes FP64 / FP32 storage only, no body force and
    the shift forcing value; its tiles are those of Guo forcing."""
    fe = dict(model=lib.LBM_MODEL_FE, kappa=0.05, gamma=0.5)
    ok = lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "f32", **fe)
    assert lib.lbm_sc_workspace_bytes(ok) > 0
    for bad in (lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "bf16", **fe),
                lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "f32", body_A=1e-5, **fe),
                lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "f32", forcing="guo", **fe),
                lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "f32", model=2),
                lib.make_params(lib.LBM_D3Q19, (8, 8, 8), 1.0, 1.0, 2.5, "f32", model=lib.LBM_MODEL_FE,
                                kappa=float("nan"), gamma=0.5)):
        assert lib.lbm_sc_workspace_bytes(bad) == 0
    h = lib.lbm_sc_create(ok, 256 * 1024, lib.lbm_sc_workspace_bytes(ok), 0)
    try:
        for t in range(len(lib.TILES)):
            good = lib.tile_supported(t, lib.LBM_D3Q19, lib.LBM_F32, 0, lib.LBM_MODEL_FE)
            assert good == (lib.TILE_KIND[t] in (0, 3) or t == 34)
            assert not (good and lib.TILE_KIND[t] == lib.RETIRED)
            if good and lib.TILE_KIND[t] in (0, 3):
                lib.lbm_sc_set_tuning(h, t, 0)
            elif not good:
                with pytest.raises(lib.LbmError):
                    lib.lbm_sc_set_tuning(h, t, 0)
    finally:
        lib.lbm_sc_destroy(h)


def test_pfm_library_exports_and_layout(lib, tmp_path):
    """libpfm.so loads without a GPU, exports every pfm_ entry point of
    include/pfm.h, its parameter struct has the C layout, and the workspace size
    validates the parameters."""
    import subprocess
    from paper_1112_5547_gb300 import phase_field as pf
    src = open(os.path.join(ROOT, "include", "pfm.h")).read()
    declared = set(re.findall(r"\b(pfm_\w+)\s*\(", re.sub(r"/\*.*?\*/", "", src, flags=re.S)))
    assert declared == set(pf.EXPORTS)
    so = ctypes.CDLL(pf.PFM_LIB)
    for name in declared:
        assert hasattr(so, name), name
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pfm.h"', "int main(void) {",
             'printf("size %zu\\n", sizeof(pfm_params));']
    for field, _ in pf.pfm_params._fields_:
        lines.append('printf("%s %%zu\\n", offsetof(pfm_params, %s));' % (field, field))
    lines.append("return 0; }")
    (tmp_path / "l.c").write_text("\n".join(lines))
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(tmp_path / "l"), str(tmp_path / "l.c")],
                   check=True)
    got = dict(x.split() for x in subprocess.run([str(tmp_path / "l")], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(pf.pfm_params)
    for field, _ in pf.pfm_params._fields_:
        assert int(got[field]) == getattr(pf.pfm_params, field).offset, field
    ok = pf.make_params((16, 20, 24), 1.4, 0.6, 0.3, 0.1, "f32")
    n = pf.workspace_bytes(ok)
    R, C = 16 * 20 * 24, 16 * 20 * 13
    assert n >= (8 * C * 2 + 8 * C * 2 + 8 * R + 11 * R + 11 * C * 2) * 4  # state, transform batches
    for bad in (pf.make_params((16, 20, 24), 1.4, 0.5, 0.3, 0.1), pf.make_params((16, 20, 24), 1.4, 0.6, 0.3, 0.0),
                pf.make_params((16, 20, 24), -1.0, 0.6, 0.3, 0.1), pf.make_params((1, 20), 1.4, 0.6, 0.3, 0.1),
                pf.make_params((16, 20, 24), 1.4, 0.6, 0.0, 0.1)):
        assert pf.workspace_bytes(bad) == 0


def test_missing_libraries_fail_loudly(tmp_path):
    """The product path has no CPU fallback: loading a library that is not there
    raises instead of degrading."""
    from paper_1112_5547_gb300 import lbm_sc, phase_field
    for mod, name in ((lbm_sc, "liblbm_sc.so"), (phase_field, "libpfm.so")):
        saved = mod._lib
        mod._lib = None
        try:
            with pytest.raises(ImportError):
                mod.load(str(tmp_path / name))
        finally:
            mod._lib = saved


def test_tuning_cache_keys_separate_the_collisions(lib):
    """The autotuner's cache keeps the SC shift, Guo and FE entries of one size apart
    (a shape tuned for one collision must not overwrite another's)."""
    from paper_1112_5547_gb300 import autotune

    class Fake:
        def __init__(self, **kw):
            self.params = lib.make_params(lib.LBM_D3Q19, (64, 64, 64), 1.0, 1.0, 2.0, "f32", **kw)
            self.lattice = lib.LBM_D3Q19
            self.shape = (64, 64, 64)
    keys = {autotune.cache_key(Fake()), autotune.cache_key(Fake(forcing="guo")),
            autotune.cache_key(Fake(model=lib.LBM_MODEL_FE, kappa=0.05, gamma=1.0))}
    assert keys == {"D3Q19/f32/64x64x64", "D3Q19/f32/64x64x64/guo", "D3Q19/f32/64x64x64/fe"}


def test_batch_tile_rule_mirror_matches_the_library(lib):
    """The binding's batch_tile_fits (used by the autotuner and the server)
    gives the library's answer (a batch workspace size above zero) for every
    batch tile, on lattices of both kinds, every storage precision, a range of
    sizes, and the forcing schemes and models the TMA tiles exclude."""
    import types
    shapes = [(8, 8, 8), (16, 8, 32), (16, 12, 32), (16, 8, 24), (20, 6, 64), (10, 12, 64), (9, 12, 48),
              (12, 40, 96), (8, 64, 128), (16, 16), (64, 64)]
    checked = 0
    for prec in lib.PRECISIONS:
        for shape in shapes:
            kind = lib.LBM_D3Q19 if len(shape) == 3 else lib.LBM_D2Q9
            for forcing, model in (("shift", lib.LBM_MODEL_SC), ("guo", lib.LBM_MODEL_SC),
                                   ("shift", lib.LBM_MODEL_FE)):
                p = lib.make_params(kind, shape, 1.0, 0.9, 2.0, prec, forcing=forcing, model=model, gamma=0.5)
                ws = lib.lbm_sc_workspace_bytes(p)
                if ws == 0:  # a combination the library does not take (the FE model stores FP32 / FP64 only)
                    assert model == lib.LBM_MODEL_FE and prec not in ("f32", "f64")
                    continue
                h = lib.lbm_sc_create(p, 256 * 1024, ws, 0)
                try:
                    for t in range(len(lib.BATCH_TILES)):
                        fits = lib.lbm_sc_batch_workspace_bytes([h], t, 0) > 0
                        assert lib.batch_tile_fits(t, types.SimpleNamespace(params=p)) == fits, (prec, shape, t)
                        checked += fits
                finally:
                    lib.lbm_sc_destroy(h)
    assert checked > 100


def test_tma_box_origins_are_16_byte_aligned(lib):
    """Every tensor copy the TMA kernels issue starts its x coordinate on a
    16-byte boundary (the hardware's rule; an unaligned one is an illegal
    instruction): the population box of a tile at x0 starts at x0 + ghost_x - 16
    bytes of values and the density box of the rest-offset storages at node
    x0 + ghost_x - 2 (two floats a node), for every TMA tile (solo and batch),
    storage precision and lattice width, with the library's own geometry."""
    widths = (32, 33, 40, 48, 63, 64, 65, 70, 96, 127, 128, 130, 512)
    solo = {t for t, k in enumerate(lib.TILE_KIND) if k in (5, 6)}
    tile_x = {lib.TILES[t][0] for t in solo} | {lib.BATCH_TILES[t][0] for t in range(len(lib.BATCH_TILES))
                                                 if lib.BATCH_TILE_TMA[t]} | {x for x, _ in lib.SHAPE3}
    for prec in ("f32", "bf16", "f16", "bf16_rest", "f16_rest"):
        for nx in widths:
            p = lib.make_params(lib.LBM_D3Q19, (16, 12, nx), 1.0, 1.0, 2.0, prec)
            h = lib.lbm_sc_create(p, 256 * 1024, lib.lbm_sc_workspace_bytes(p), 0)
            try:
                e, q, px, py, gx, gy, _ = lib.lbm_sc_layout(h)
            finally:
                lib.lbm_sc_destroy(h)
            assert (px * e) % 16 == 0
            pad = 16 // e
            for tx in tile_x:
                for x0 in range(0, nx, tx):
                    assert ((x0 + gx - pad) * e) % 16 == 0, (prec, nx, tx, x0)
                    if prec.endswith("_rest"):
                        assert (2 * (x0 + gx - 2) * 4) % 16 == 0, (prec, nx, tx, x0)
