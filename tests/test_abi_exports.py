"""The C ABI: every function include/*.h declares is exported by the built
libemc.so with C linkage (loaded and looked up only; no device calls), and
the status codes and tally kinds the binding uses match the header."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?(?:emc_status|int64_t|int32_t|char\s*\*|void|double)\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                  re.M)


def declared() -> list[str]:
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += DECL.findall(src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("emc_init", "emc_batch_init", "emc_step", "emc_tally", "poisson_solve", "emc_set_temperature",
                 "emc_mlp_train", "emc_mlp_infer", "emc_thermal_solve", "emc_last_error", "emc_destroy"):
        assert must in names, must
    assert len(names) >= 25


def test_library_exports_every_declared_symbol(emc):
    lib = ctypes.CDLL(emc.emc.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_codes_and_tally_kinds_match_header(emc):
    h = open(os.path.join(ROOT, "include", "emc.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(EMC_[A-Z0-9_]+)\s*=\s*(\d+)", h))
    assert codes["EMC_OK"] == 0
    for name in ("TALLY_OBS", "TALLY_EVENTS", "TALLY_HEAT", "TALLY_CHARGE", "TALLY_CROSSINGS", "TALLY_PHI",
                 "TALLY_FIELD", "TALLY_HEAT_J", "TALLY_EVENTS_CELL"):
        assert getattr(emc, name) == codes["EMC_" + name], name
    assert emc.FP32 == codes["EMC_FP32"] and emc.FP64 == codes["EMC_FP64"]
    assert emc.GEOM_BULK == codes["EMC_GEOM_BULK"] and emc.GEOM_NANOWIRE == codes["EMC_GEOM_NANOWIRE"]


def test_config_struct_layout_matches_header(emc):
    """The ctypes mirror of emc_config lists the header's fields in order."""
    h = open(os.path.join(ROOT, "include", "emc.h")).read()
    body = h[h.index("typedef struct emc_config {"):h.index("} emc_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for line in body.splitlines()[1:]:
        m = re.match(r"\s*(?:double|int64_t|int32_t|uint32_t)\s+(.+);", line)
        if m:
            fields += [re.sub(r"\[.*\]", "", f).strip() for f in m.group(1).split(",")]
    assert [f for f, _ in emc.EmcConfig._fields_] == fields
