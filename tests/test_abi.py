"""The C-ABI library builds, loads without a GPU, and exports every symbol the header declares.

No compute call is made here: only entry points that touch no device
(bundle_default_params, bundle_status_string, bundle_last_error) run, which is
enough to check the ctypes mirror of bundle_params field by field.
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bundle.h")


@pytest.fixture(scope="module")
def built():
    from paper_1504_02687_gb300 import build

    return build.build()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bundle_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bundle_init", "bundle_init_polylines", "bundle_iterate", "bundle_fetch",
                 "bundle_fetch_density", "bundle_destroy", "bundle_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(bundle_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    import paper_1504_02687_gb300 as pkg

    assert set(pkg.EXPORTED) == set(_declared())


def test_library_loads_and_params_mirror_matches(built):
    import paper_1504_02687_gb300 as pkg

    p = pkg.default_params()
    assert (p.grid_w, p.grid_h, p.grid_dominant, p.margin_px) == (0, 0, 800, -1)
    assert (p.radius, p.passes, p.alpha_num, p.alpha_den) == (4, 3, 1, 4)
    assert p.h_max_sigmas == 2.0 and abs(p.lambda_ - 0.9) < 1e-15
    assert (p.n_fixed, p.n_max) == (0, 64)
    assert p.delta_px == 2.0 and p.laplace_beta == 0.5 and abs(p.eps - 1e-9) < 1e-15
    assert (p.step_tries, p.sum_bits, p.rho_dtype, p.flags) == (8, 0, 0, 0)
    assert pkg.status_string(pkg.BUNDLE_EOVERFLOW) == "BUNDLE_EOVERFLOW"


def test_struct_mirrors_match_the_c_layout(tmp_path):
    """Compile a probe against the header and compare every field offset with ctypes."""
    import paper_1504_02687_gb300 as pkg

    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    pairs = (("bundle_params", pkg.BundleParams), ("bundle_info", pkg.BundleInfo),
             ("bundle_graph_desc", pkg.BundleGraphDesc),
             ("bundle_render_params", pkg.BundleRenderParams))
    for cname, cls in pairs:
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, cls in pairs:
        assert int(got[cname]) == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_init_without_gpu_fails_cleanly(built):
    """With no device the library reports an error status; it never falls back to the CPU."""
    import numpy as np
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1504_02687_gb300 as pkg

    src = np.zeros((4, 2), np.float32)
    dst = np.ones((4, 2), np.float32)
    with pytest.raises(pkg.BundleError) as ei:
        pkg.bundle_init(pkg.default_params(grid_w=64, grid_h=64), src, dst)
    assert ei.value.status in (pkg.BUNDLE_ECUDA, pkg.BUNDLE_ENOMEM)


def test_binding_constants_match_the_header():
    """Every #define and status value the binding mirrors has the header's value."""
    import paper_1504_02687_gb300 as pkg

    txt = open(HEADER).read()
    defs = {m.group(1): int(m.group(2))
            for m in re.finditer(r"^#define (BUNDLE_[A-Z_0-9]+) (\d+)", txt, flags=re.M)}
    pairs = {"BUNDLE_FLAG_FIXED_STEP": pkg.FLAG_FIXED_STEP,
             "BUNDLE_FLAG_SEGMENT_HIST": pkg.FLAG_SEGMENT_HIST,
             "BUNDLE_FLAG_INK_STATS": pkg.FLAG_INK_STATS,
             "BUNDLE_FLAG_LOAD_GATHERS": pkg.FLAG_LOAD_GATHERS,
             "BUNDLE_INPUT_DEVICE": pkg.INPUT_DEVICE,
             "BUNDLE_FETCH_DEVICE": pkg.FETCH_DEVICE,
             "BUNDLE_FETCH_PIXELS": pkg.FETCH_PIXELS,
             "BUNDLE_FETCH_RESAMPLED": pkg.FETCH_RESAMPLED,
             "BUNDLE_DENSITY_HIST": pkg.DENSITY_HIST,
             "BUNDLE_DENSITY_SUMS": pkg.DENSITY_SUMS,
             "BUNDLE_DENSITY_RHO": pkg.DENSITY_RHO,
             "BUNDLE_INK_STATS_CAP": pkg.INK_STATS_CAP,
             "BUNDLE_PROFILE_KINDS": len(pkg.PROFILE_KINDS),
             "BUNDLE_STEP_LAST": pkg.STEP_LAST}
    for name, value in pairs.items():
        assert defs[name] == value, name
    # the flags are distinct bits
    flags = [v for k, v in defs.items() if k.startswith("BUNDLE_FLAG_")]
    assert len(flags) == len(set(flags)) and all(f & (f - 1) == 0 for f in flags)
    # status and density-type enums
    for name in ("BUNDLE_OK", "BUNDLE_EINVAL", "BUNDLE_ENOMEM", "BUNDLE_ECUDA", "BUNDLE_EOVERFLOW",
                 "BUNDLE_ETIMEOUT", "BUNDLE_ESTATE", "BUNDLE_ENOTSUP"):
        m = re.search(rf"\b{name} = (\d+)", txt)
        assert m and int(m.group(1)) == getattr(pkg, name), name
    for name, attr in (("BUNDLE_RHO_F32", "RHO_F32"), ("BUNDLE_RHO_BF16", "RHO_BF16"),
                       ("BUNDLE_RHO_F16", "RHO_F16")):
        m = re.search(rf"\b{name} = (\d+)", txt)
        assert m and int(m.group(1)) == getattr(pkg, attr), name
