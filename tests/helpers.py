"""Shared test helpers: loading a synthetic model into the CUDA library and comparing
results with the oracle."""
import numpy as np


def rel_err(a, b, floor=0.0):
    """The paper's relative difference 2|a-b|/(|a|+|b|) (Sec. 4.1.1), elementwise."""
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    den = np.abs(a) + np.abs(b)
    out = np.zeros(np.broadcast(a, b).shape)
    nz = den > floor
    out[nz] = 2.0 * np.abs(a - b)[nz] / den[nz]
    return out


def gpu_context(model, oracle_dirs=None, **opts):
    """A library context holding the model. When oracle_dirs is given, the GPU uses the
    same direction vectors as the oracle (required for bit-exact ray comparisons)."""
    import paper_1912_08445_gb300 as mg
    ctx = mg.Context(**opts)
    ctx.load_model(model, dirs=oracle_dirs)
    return ctx


def compare_rays(ctx, tr, origins, R):
    """Bit-exact comparison of GPU half-rays with the oracle's trace_all output."""
    bad = []
    for io, o in enumerate(origins):
        for r in range(R):
            k = io * R + r
            s, e = tr["off"][k], tr["off"][k + 1]
            g = ctx.get_ray(o, r)
            ok = (np.array_equal(g["cells"], tr["cells"][s:e]) and np.array_equal(g["nsub"], tr["nsub"][s:e])
                  and np.array_equal(g["ds"].view(np.uint64), tr["ds"][s:e].view(np.uint64))
                  and np.array_equal(g["vpar"].view(np.uint64), tr["vpar"][s:e].view(np.uint64)))
            if not ok:
                bad.append((int(o), r))
    return bad
