"""Small, self-contained profiling case: one function, one form, a few calls.

    python -m paper_2605_15547_gb300.profile_case expf df 25 3 [variant]

evaluates `func` in `form` on 2^log2n inputs (uniform domain bit patterns; binary64:
the paper's U[-20,20] / U[0.125,8]) `reps` times, with the main kernel's launch shape
`variant` (default: the library's default shape).  Used as the command profiled by ncu
(sized to stay a few hundred MB on the device).
"""
import sys

import numpy as np
import torch

import paper_2605_15547_gb300 as crm
from paper_2605_15547_gb300 import workloads as W


def main(argv):
    func = argv[1] if len(argv) > 1 else "expf"
    form = argv[2] if len(argv) > 2 else "df"
    log2n = int(argv[3]) if len(argv) > 3 else 25
    reps = int(argv[4]) if len(argv) > 4 else 3
    if len(argv) > 5:
        crm.set_variant(func, int(argv[5]), form=form)
    n = 1 << log2n
    if func in W.F32_FUNCS:
        x = W.domain_bits(func, n, W.rng_for(2, func)).view(np.float32)
    else:
        x = W.f64_uniform(-20, 20, n, W.rng_for(5, func)) if func == "exp2" else \
            W.f64_uniform(0.125, 8.0, n, W.rng_for(5, func))
    xd = torch.from_numpy(x).cuda()
    y = crm.eval(func, xd, form=form)
    for _ in range(reps):
        crm.eval_into(func, xd, y, form=form)
    torch.cuda.synchronize()
    print("ok", func, form, n, crm.get_variant(func, form=form), crm.stats())


if __name__ == "__main__":
    main(sys.argv)
