"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol that
include/sphc.h declares."""
import ctypes
import os
import re

import paper_2506_08284_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sphc.h")).read()
    return sorted(set(re.findall(r"SPHC_API\s+[\w\s\*]*?\b(sphc_\w+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_symbols()
    for n in ["sphc_setup", "sphc_solve", "sphc_destroy", "sphc_last_error", "sphc_export"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = pkg.sphc.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(pkg.sphc.EXPORTED)


def test_default_options_without_gpu():
    o = pkg.sphc.default_opts()
    assert (o.max_levels, o.emin_iters, o.max_coarse, o.emin_omega, o.vcycle_fp32) == (8, 1, 1000, 0.5, 1)
    assert o.power_iters == 15 and o.max_iter == 500
    assert (o.cg_graph, o.learned, o.learned_emin_iters, o.autotune, o.sweep_form) == (1, 0, 0, 0, 0)
    assert pkg.sphc.load().sphc_default_opts(None) == -1


def test_option_and_info_structs_match_the_header():
    # the ctypes mirrors of sphc_opts and sphc_level_info list the header's fields in its order
    text = open(os.path.join(ROOT, "include", "sphc.h")).read()

    def fields(struct):
        end = re.search(r"\}\s*" + struct + ";", text).start()
        body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                m = re.search(r"(\w+)\s*(\[\w+\])?\s*$", part.strip())
                names.append(m.group(1))
        return names

    assert fields("sphc_opts") == [f[0] for f in pkg.sphc.sphc_opts._fields_]
    assert fields("sphc_level_info") == [f[0] for f in pkg.sphc.sphc_level_info._fields_]
