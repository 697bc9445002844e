"""Run a named synthetic workload for a number of steps and print its statistics (JSON).

    python -m paper_2403_11156_gb300.run_scene --scene rigid --steps 2 --eager

Workloads: small (8k-particle dam break), rigid (1.2M-particle dam break with rigid boxes),
column (250k-particle high-viscosity column), batch (64 dam breaks of 20k-200k particles),
wcsph (the 8k dam break under the equation-of-state solver).
--eager launches the kernels one by one (the form a kernel profiler can attribute);
without it a step is one CUDA-graph launch.  --lanes sets the threads per particle of the
neighbour sweeps (1, 2, 4, 8; 0 chooses by size).  --surface / --image write the post-processing
results of scene 0 after the steps: the iso-surface of the fluid (OBJ) and a shaded
height map seen from above (PGM).  --warm picks the warm start of the solves (zero,
previous, learned); the learned one loads a parameter block (--mlp, .npy) or, without one,
first trains the network on 50k solver states of a seeded 0.5M-particle dam break.
"""
from __future__ import annotations

import argparse
import json
import time

from paper_2403_11156_gb300 import build, scenes, sph

WORKLOADS = {
    "small": lambda: [scenes.dam_break_small()],
    "rigid": lambda: [scenes.dam_break_rigid()],
    "column": lambda: [scenes.viscous_column()],
    "batch": lambda: scenes.batch_dam_break(),
    "wcsph": lambda: [scenes.dam_break_wcsph()],
}
WARM = {"zero": scenes.WARM_ZERO, "previous": scenes.WARM_PREVIOUS, "learned": scenes.WARM_LEARNED}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", default="rigid", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--eager", action="store_true")
    ap.add_argument("--dt", type=float, default=0.0)
    ap.add_argument("--lanes", type=int, default=0, help="threads per particle (0: by size)")
    ap.add_argument("--surface", default=None, help="write the fluid's iso-surface (OBJ) of scene 0 here")
    ap.add_argument("--image", default=None, help="write a height-map image (PGM) of scene 0 here")
    ap.add_argument("--grid", type=float, default=0.0, help="surface grid spacing (default: r)")
    ap.add_argument("--warm", default=None, choices=sorted(WARM), help="warm start (default: the workload's)")
    ap.add_argument("--mlp", default=None, help="network parameter block (.npy) for --warm learned")
    args = ap.parse_args()
    build.build()
    params = None
    if args.warm == "learned":
        import numpy as np
        if args.mlp:
            params = np.load(args.mlp)
        else:
            from paper_2403_11156_gb300 import warmstart
            f, y = warmstart.generate_dataset(50_000, 50, n_scenes=1, size_range=(5e5, 5e5))
            params, _ = warmstart.train(f, y, epochs=30)
    descs = WORKLOADS[args.scene]()
    for d in descs:
        d["lanes_per_particle"] = args.lanes
        if args.warm:
            d["warm_start"] = WARM[args.warm]
    g = sph.Context(descs, torch_allocator=False)
    if params is not None:
        g.sph_set_mlp(params)
    g.sph_set_mode(graph=not args.eager, timing=False)
    t = time.perf_counter()
    g.sph_steps(args.steps, args.dt)
    status = g.sph_synchronize(raise_on_error=False)
    el = time.perf_counter() - t
    out = {"scene": args.scene, "scenes": len(descs), "steps": args.steps,
           "fluid_particles": int(sum(len(d["fluid_x"]) for d in descs)),
           "seconds": el, "status": sph.STATUS_NAMES[status], "stats": g.sph_get_stats(0)}
    d0 = descs[0]
    if args.surface:
        # post-processing (Sec. 4.3): the volume-fraction field's 0.5 iso-surface
        from paper_2403_11156_gb300 import export
        s = args.grid or d0["radius"]
        lo, hi = d0["domain_min"], d0["domain_max"]
        dims = [int((hi[a] - lo[a]) / s) + 1 for a in range(3)]
        field = g.sph_surface_field(lo, s, dims)
        tris = sph.sph_surface_mesh(field, lo, s, 0.5)
        out["surface"] = {"path": args.surface, "triangles": int(len(tris)),
                          "vertices": export.write_obj(tris, args.surface)}
    if args.image:
        from paper_2403_11156_gb300 import export
        lo, hi = d0["domain_min"], d0["domain_max"]
        px = d0["radius"] / 2
        w, h = int((hi[0] - lo[0]) / px), int((hi[1] - lo[1]) / px)
        hm = g.sph_render_heightmap(lo[:2], (lo[0] + w * px, lo[1] + h * px), w, h, d0["radius"])
        export.write_pgm(hm, px, args.image)
        out["image"] = {"path": args.image, "width": w, "height": h}
    print(json.dumps(out))
    g.close()


if __name__ == "__main__":
    main()
