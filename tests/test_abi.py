"""CPU checks of the C ABI: the library builds, loads without a GPU, exports every entry point
that include/dass.h declares, and rejects bad arguments on the host before any launch."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dass.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(dass_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_14847_gb300 import build, dass
    build.ensure_built()
    return dass.load()


def test_header_declares_the_hot_path():
    names = declared()
    for required in ("dass_preprocess", "dass_bin_sort", "dass_render_fwd", "dass_render_bwd", "dass_shift",
                     "dass_densify_stats", "dass_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2411_14847_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(dass_\w+)\b", out))
    for name in declared():
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing else leaks out of the library but the dass_ entry points
    others = [l.split()[-1] for l in out.splitlines() if " T " in l and "dass_" not in l]
    assert not [o for o in others if not o.startswith("_")], others


def test_binding_covers_header():
    from paper_2411_14847_gb300 import dass
    assert sorted(dass.exported_symbols()) == declared()


def test_host_side_argument_checks(lib):
    from paper_2411_14847_gb300 import dass, synth
    assert lib.dass_version() == 1
    assert lib.dass_status_string(-4) == b"capacity exceeded"
    cams = dass.cameras(synth.arc_cameras(2, 4.0, 100, 50))
    t, p = C.c_int32(), C.c_int64()
    assert lib.dass_tile_layout(cams, 2, 16, C.byref(t), C.byref(p)) == 0
    assert (t.value, p.value) == (2 * 7 * 4, 2 * 5000)
    assert lib.dass_tile_layout(cams, 2, 12, C.byref(t), C.byref(p)) == -1          # unsupported tile
    assert lib.dass_tile_layout(cams, 65, 16, C.byref(t), C.byref(p)) == -1         # too many cameras
    # bad sizes/NULLs are rejected before anything touches the device
    assert lib.dass_preprocess(-1, 0, None, None, None, None, None, None, cams, 2, 16, None, None) == -1
    assert lib.dass_preprocess(10, 4, None, None, None, None, None, None, cams, 2, 16, None, None) == -1
    assert lib.dass_render_fwd(None, None, None, cams, 2, 16, 100, None, None, None, None, None, None) == -1
    assert lib.dass_tile_order(None, 5, None, None) == -1                            # missing buffers
    assert lib.dass_tile_order(None, 0, None, None) == 0                             # no tiles: a no-op
    assert lib.dass_shift(-5, None, None, None, None, None, None, None) == -1
    assert lib.dass_densify_select(10, None, None, None, None, 1e-4, -1.0, 10, None, None, None, 0, None) == -1
    b = C.c_size_t()
    assert lib.dass_bin_sort_workspace(1000, 5000, 10, C.byref(b)) == 0 and b.value > 0
    # pair positions are int32 in the compositing kernels: capacities of 2^31 or more are refused
    assert lib.dass_bin_sort_workspace(1000, (1 << 31) - 1, 10, C.byref(b)) == 0
    assert lib.dass_bin_sort_workspace(1000, 1 << 31, 10, C.byref(b)) == -1
    # a workspace smaller than the query is reported as DASS_ERR_OOM
    fake = C.c_void_p(16)
    assert lib.dass_bin_sort(fake, 10, cams, 2, 16, fake, 100, fake, fake, fake, 8, None) == -3
    assert lib.dass_bin_sort(fake, 10, cams, 2, 16, fake, 1 << 31, fake, fake, fake, 1 << 40, None) == -1
    assert lib.dass_bin_sort_static(fake, 10, cams, 2, 16, fake, 1 << 31, fake, fake, None) == -1
    # empty inputs are no-ops that succeed without launching
    assert lib.dass_shift(0, None, None, None, None, None, None, None) == 0
    assert lib.dass_preprocess(0, 0, None, None, None, None, None, None, cams, 2, 16, None, None) == 0


def test_host_side_layout_checks(lib):
    """Cameras whose planes would overflow 32-bit pixel offsets, and feature rows that are not
    16-byte aligned (they are read as float4), are rejected before any launch."""
    from paper_2411_14847_gb300 import dass, synth
    t, p = C.c_int32(), C.c_int64()
    big = synth.arc_cameras(1, 4.0, 50000, 50000)
    assert lib.dass_tile_layout(dass.cameras(big), 1, 16, C.byref(t), C.byref(p)) == -1
    ok = synth.arc_cameras(1, 4.0, 40000, 40000)
    assert lib.dass_tile_layout(dass.cameras(ok), 1, 16, C.byref(t), C.byref(p)) == 0
    aligned, misaligned = C.c_void_p(256), C.c_void_p(260)
    assert lib.dass_object_ids(misaligned, 10, 16, aligned, aligned, 4, aligned, None) == -1
    assert lib.dass_object_ids(aligned, 10, 16, misaligned, aligned, 4, aligned, None) == -1
    assert lib.dass_dynamic_gaussians(misaligned, 10, 16, aligned, aligned, 4, aligned, aligned, None) == -1
    cams = dass.cameras(synth.arc_cameras(2, 4.0, 100, 50))
    assert lib.dass_render_features(aligned, aligned, aligned, cams, 2, 16, misaligned, 16, 10, aligned, None) == -1
    assert lib.dass_render_features(aligned, aligned, aligned, cams, 2, 16, aligned, 16, 1 << 31, aligned, None) == -1


def test_host_side_field_and_loss_checks(lib):
    """Deformation-field descriptors and the cached-loss statistics are validated on the host:
    a malformed field is refused, an empty row set succeeds without a launch, a (levels,
    features) shape without a compiled kernel reports DASS_ERR_UNSUPPORTED before launching,
    and misaligned statistics pairs are refused."""
    from paper_2411_14847_gb300 import dass, synth
    f = dass.dass_field()
    f.levels, f.features, f.log2_table, f.hidden = 16, 2, 14, 64
    for i in range(16):
        f.res[i] = 16 + i
    for d in range(3):
        f.bbox_min[d], f.bbox_max[d] = -1.0, 1.0
    for k in ("table", "w1", "b1", "w2", "b2"):
        setattr(f, k, 256)
    ok = C.c_void_p(256)
    assert lib.dass_field_fwd(C.byref(f), 0, None, ok, ok, None) == 0          # empty: no launch
    assert lib.dass_field_fwd(C.byref(f), -1, None, ok, ok, None) == -1
    bad = dass.dass_field.from_buffer_copy(f)
    bad.features = 3
    assert lib.dass_field_fwd(C.byref(bad), 5, None, ok, ok, None) == -1      # features not in {2, 4}
    bad = dass.dass_field.from_buffer_copy(f)
    bad.hidden = 32
    assert lib.dass_field_fwd(C.byref(bad), 5, None, ok, ok, None) == -1      # hidden width fixed at 64
    odd = dass.dass_field.from_buffer_copy(f)
    odd.levels = 12
    assert lib.dass_field_fwd(C.byref(odd), 5, None, ok, ok, None) == -6      # no kernel for 12 levels
    cams = dass.cameras(synth.arc_cameras(2, 4.0, 100, 50))
    assert lib.dass_loss_target_stats(ok, cams, 2, C.c_void_p(260), None) == -1
    assert lib.dass_loss_cached(ok, ok, C.c_void_p(260), cams, 2, C.c_float(0.2), ok, ok, ok, 1 << 30, None) == -1
    assert lib.dass_loss_cached(ok, ok, ok, cams, 2, C.c_float(1.5), ok, ok, ok, 1 << 30, None) == -1   # lambda


def test_struct_layouts_match_the_header(tmp_path):
    """Every descriptor the binding passes by pointer has the header's layout: a C program built
    with the system compiler prints sizeof and each field's offsetof, compared with ctypes."""
    import ctypes as C
    from paper_2411_14847_gb300 import dass
    structs = [dass.dass_camera, dass.dass_scene, dass.dass_step_desc, dass.dass_inherit_step_desc,
               dass.dass_densify_step_desc, dass.dass_timestep_desc, dass.dass_timestep_stats, dass.dass_field]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dass.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("{s.__name__} %zu\\n", sizeof({s.__name__}));')
        for f, _ in s._fields_:
            lines.append(f'printf("{s.__name__}.{f} %zu\\n", offsetof({s.__name__}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for s in structs:
        assert int(got[s.__name__]) == C.sizeof(s), s.__name__
        for f, _ in s._fields_:
            assert int(got[f"{s.__name__}.{f}"]) == getattr(s, f).offset, (s.__name__, f)


def test_timestep_descriptor_prefetch_checks(lib):
    """dass_timestep refuses, on the host and before any device work, a descriptor whose prefetch
    fields are half set or whose prefetch buffer overlaps the targets. The same descriptor without them, or with
    both set to a separate buffer, passes the checks and stops at the workspace size (DASS_ERR_OOM),
    still on the host. The pointers are stand-ins that the host checks never dereference."""
    from paper_2411_14847_gb300 import dass, synth
    cams = dass.cameras(synth.arc_cameras(2, 4.0, 100, 50))
    n_host = C.c_int64(100)
    bufs = [C.create_string_buffer(64) for _ in range(12)]

    def ptr(i):
        return C.cast(bufs[i], C.c_void_p).value

    d = dass.dass_timestep_desc()
    d.n_max, d.sh_degree, d.n_cams = 200, 1, 2
    d.means, d.log_scales, d.quats, d.opacity_logit, d.sh, d.is_var = (ptr(i) for i in range(6))
    d.n, d.cams = C.cast(C.pointer(n_host), C.c_void_p), C.cast(cams, C.c_void_p)
    d.targets, d.offsets, d.z, d.workspace = ptr(6), ptr(7), ptr(8), ptr(9)
    d.workspace_bytes = 16
    d.tile, d.batch, d.pair_capacity, d.k_max = 16, 128, 1 << 16, 10
    d.lambda_dssim, d.quantile, d.prune_opacity = 0.2, 0.5, 0.005
    stats = dass.dass_timestep_stats()

    def call():
        return lib.dass_timestep(C.byref(d), C.byref(stats), None)

    assert call() == dass.ERR_OOM
    # the targets hold 2 x 100 x 50 x 3 floats from ptr(6); the prefetch buffers are addresses relative
    # to it (only compared, never dereferenced): half set, the targets themselves, one starting inside
    image = 4 * 100 * 50 * 3 * 2
    for nh, nd in ((ptr(10), None), (None, ptr(6) + 4 * image), (ptr(10), ptr(6)), (ptr(10), ptr(6) + image - 4),
                   (ptr(10), ptr(6) - image + 4)):
        d.next_targets_host, d.next_targets = nh, nd
        assert call() == dass.ERR_INVALID_ARG, (nh, nd)
    for nd in (ptr(6) + image, ptr(6) + 4 * image, ptr(6) - image):    # adjacent or apart
        d.next_targets_host, d.next_targets = ptr(10), nd
        assert call() == dass.ERR_OOM, nd
