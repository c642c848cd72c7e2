"""The C-ABI library without a GPU: it loads, exports every symbol its header
declares, derives the Radau constants the kernels use (checked against the
oracle's independent derivation) and validates arguments on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O
from paper_1607_03884_gb300 import kin, synth


def header_functions():
    txt = open(os.path.join(ROOT, "include", "kin.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kin_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = kin.lib()
    names = header_functions()
    assert set(names) == set(kin.EXPORTS)
    for name in names:
        assert hasattr(L, name), name


def test_radau_constants_match_oracle_derivation():
    g = kin.radau_constants()
    tb = O.tableau()
    np.testing.assert_allclose(g["c"], tb["c"], rtol=0, atol=1e-15)
    np.testing.assert_allclose([g["gamma"], g["alpha"], g["beta"]],
                               [tb["gamma"], tb["alpha"], tb["beta"]], rtol=1e-14)
    np.testing.assert_allclose(g["T"], tb["T"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["TI"], tb["TI"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(g["d"], tb["e"] / tb["gamma0"], rtol=1e-13)


def test_options_defaults():
    o = kin.options()
    assert (o.layout, o.lu_fp32, o.jac_fd, o.max_steps, o.nit, o.transform_tol) == (3, 0, 0,
                                                                                     100000, 7, 1)
    assert kin.lib().kin_options_default(None) == kin.KIN_ERR_INVALID_ARG


def _desc(mech, **over):
    arrs = dict(W=mech.W, nasa=mech.nasa, reac=mech.reac.astype(np.int32),
                prod=mech.prod.astype(np.int32), arrh=mech.arrh,
                rtype=mech.rtype.astype(np.int32), eff=mech.eff, fall=mech.fall)
    arrs.update(over)
    arrs = {k: np.ascontiguousarray(v) for k, v in arrs.items()}
    d = kin.MechDesc(mech.ns, mech.nr, *(arrs[k].ctypes.data for k in
                                          ("W", "nasa", "reac", "prod", "arrh", "rtype", "eff",
                                           "fall")))
    return d, arrs


def _create(d):
    h = C.c_void_p()
    return kin.lib().kin_mech_create(C.byref(d), C.byref(h))


def test_mech_create_rejects_bad_descriptions(h2_mech):
    L = kin.lib()
    assert L.kin_mech_create(None, None) == kin.KIN_ERR_INVALID_ARG
    reac = h2_mech.reac.astype(np.int32).copy()
    reac[0, 0] = h2_mech.ns           # out of range
    assert _create(_desc(h2_mech, reac=reac)[0]) == kin.KIN_ERR_MECH
    reac = h2_mech.reac.astype(np.int32).copy()
    reac[0, 0] = h2_mech.ns - 1       # the inert must not react
    assert _create(_desc(h2_mech, reac=reac)[0]) == kin.KIN_ERR_MECH
    W = h2_mech.W.copy()
    W[2] = 0.0
    assert _create(_desc(h2_mech, W=W)[0]) == kin.KIN_ERR_MECH
    rt = h2_mech.rtype.astype(np.int32).copy()
    rt[0] = 7
    assert _create(_desc(h2_mech, rtype=rt)[0]) == kin.KIN_ERR_MECH
    d, _ = _desc(h2_mech)
    d.ns = kin.MAX_SPECIES + 1
    assert _create(d) == kin.KIN_ERR_INVALID_ARG
    d.ns = 1
    assert _create(d) == kin.KIN_ERR_INVALID_ARG


def test_integrate_rejects_bad_arguments():
    L = kin.lib()
    buf = np.zeros(16)
    p = buf.ctypes.data
    # NULL mechanism
    assert L.kin_integrate(None, p, p, p, 4, 1e-6, 1e-6, 1e-10, None) == kin.KIN_ERR_INVALID_ARG
    assert L.kin_integrate_host(None, p, p, p, 4, 1e-6, 1e-6, 1e-10, None, None, None,
                                None) == kin.KIN_ERR_INVALID_ARG
    assert L.kin_get_stats(None, p) == kin.KIN_ERR_INVALID_ARG
    assert L.kin_radau_constants(p, 5) == kin.KIN_ERR_INVALID_ARG
    assert kin.lib().kin_status_string(kin.KIN_ERR_MECH) == b"invalid mechanism description"


def test_order_states_validates_on_host():
    L = kin.lib()
    assert L.kin_order_states(None, None, None, None, 4, 1e-6, 1e-10, 1, None, None,
                              None) == kin.KIN_ERR_INVALID_ARG
    o = kin.options()
    assert o.order is None


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/kin.h, from gcc."""
    import subprocess
    import tempfile
    body = "\n".join(f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = f"""#include <stddef.h>
#include <stdio.h>
#include "kin.h"
int main(void) {{
  printf("%zu\\n", sizeof({struct}));
{body}
  return 0;
}}
"""
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("ctype,cname", [(kin.Options, "kin_options"), (kin.MechDesc, "kin_mech_desc")])
def test_binding_structs_match_the_header_layout(ctype, cname):
    names = [f[0] for f in ctype._fields_]
    size, offs = _c_layout(cname, names)
    assert size == C.sizeof(ctype)
    assert offs == [getattr(ctype, n).offset for n in names]
