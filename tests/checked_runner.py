"""Runs small RACIPE cases through whichever library GRINS_RACIPE_LIB selects
and saves the results; with the index-checked build it also reports the first
recorded index/alignment violation (0 = none).  Used by test_zz_checked_build.py
in a subprocess so that the checked library is never mixed with the release one."""
import ctypes as C
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2503_18356_gb300 import api, workloads as W  # noqa: E402

CASES = {
    "ts": (W.toggle_switch(), 40, 20),
    "net5": (W.random_network(1001, 5, 10, 5, 0), 60, 20),
    "net22": (W.random_network(1002, 22, 82, 33, 3), 40, 10),
    "n30": (W.density_network(11, 30, 0.1), 8, 4),
}


def main(out_path, which):
    checked = "checked" in os.environ.get("GRINS_RACIPE_LIB", "")
    res = {}
    codes = {}
    for name in which:
        topo, S, I = CASES[name]
        h = api.Racipe.from_topology(topo)
        params, ic = h.sample_params(7, S, I)
        for prec in (1, 0):
            for polish in (1, 0):
                o = h.integrate(params, ic, precision=prec, polish=polish,
                                t_grid=np.linspace(0, 10, 6) if polish == 0 else None)
                sid, nu = h.unique_states(params, o["states"], o["status"])
                torch.cuda.synchronize()
                key = "%s_p%d_pol%d" % (name, prec, polish)
                res[key + "_states"] = o["states"].cpu().numpy()
                res[key + "_status"] = o["status"].cpu().numpy()
                res[key + "_nu"] = nu.cpu().numpy()
        if checked:
            f = api._lib.grins_debug_check_status
            f.restype = C.c_int
            f.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
            info = C.c_longlong(0)
            codes[name] = (f(h._h, C.byref(info)), info.value)
            # the no-allocation entry point writes its check words into the
            # library's static array, read by their own accessor
            N = topo.n_nodes
            buf = dict(states=torch.empty((S, I, N), dtype=torch.float64, device=params.device),
                       status=torch.empty((S, I), dtype=torch.uint8, device=params.device),
                       t_final=torch.empty((S, I), dtype=torch.float64, device=params.device),
                       err_est=torch.empty((S, I), dtype=torch.float32, device=params.device),
                       n_steps=torch.empty((S, I), dtype=torch.int32, device=params.device))
            h.integrate_static(params, ic, buf)
            torch.cuda.synchronize()
            fs = api._lib.grins_debug_static_check_status
            fs.restype = C.c_int
            fs.argtypes = [C.POINTER(C.c_longlong)]
            info = C.c_longlong(0)
            codes[name + "_static"] = (fs(C.byref(info)), info.value)
        h.close()
    np.savez(out_path, **res)
    print("CHECK", codes)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2:] or list(CASES))
