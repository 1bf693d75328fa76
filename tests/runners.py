"""Build an oracle run and a CUDA-library run from the same workload description."""

import numpy as np

from oracle import beam as obeam
from oracle import fsi as ofsi


def oracle_sim(w, **kw):
    from oracle import kinematics as okin
    bodies = []
    for b in w["bodies"]:
        if b["kind"] == "driven":
            kin = okin.FlappingKinematics(b["a0"], b["beta"], b["sigma_t"], b["sigma_r"], b["freq"])
            bodies.append(okin.DrivenPlate(b["ref"], b["s_lo"], b["n_pts"], w["ds"], kin))
        elif b["kind"] == "hinged":
            bodies.append(okin.HingedPlate(bodies[b["driver"]], b["l1"], b["n_pts"], w["ds"], b["inertia"],
                                           b["damping"], b["stiffness"], b["mass"], b["l2"], b["theta"]))
        elif b["kind"] == "torsional":
            bodies.append(ofsi.TorsionalBody(b["hinge"], b["theta0"], b["n_pts"], w["ds"], b["inertia"], b["damping"],
                                             b["stiffness"], b["theta"]))
        elif b["kind"] == "deformable":
            bodies.append(obeam.Beam(b["clamp"], b["theta0"], b["n_pts"] - 1, w["ds"], b["mass"], b["ei"], b["ea"],
                                     tip_angle=b["tip_angle"]))
        else:
            bodies.append(ofsi.RigidBody(b["pts"], b.get("ur"), b.get("appended", False)))
    kw.setdefault("drop_tol", w.get("drop_tol", 0.0))
    return ofsi.Sim(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["n_levels"], w["re"], w["dt"], w["uinf"],
                    w["sd_box"], bodies, w["ds"], **kw)


def gpu_context(w, precision=0, use_graph=True, precompute=True, stream=None, b0_method=0, drop_tol=None, **kw):
    if drop_tol is None:
        drop_tol = w.get("drop_tol", 0.0)     # the workload's filter of B0 (Eq. filtereq), if it names one
    import paper_2103_06415_gb300 as lib
    c = lib.Context(w["nx"], w["ny"], w["n_levels"], w["x0"], w["y0"], w["h"], w["re"], w["dt"], w["uinf"],
                    precision=precision, use_graph=use_graph, stream=stream, b0_method=b0_method, **kw)
    for b in w["bodies"]:
        if b["kind"] == "driven":
            c.add_driven(b["ref"], b["s_lo"], b["n_pts"], w["ds"], b["a0"], b["beta"], b["sigma_t"], b["sigma_r"],
                         b["freq"])
        elif b["kind"] == "hinged":
            c.add_torsional((0.0, 0.0), 0.0, b["n_pts"], w["ds"], b["inertia"], b["damping"], b["stiffness"],
                            b["theta"], driver=b["driver"], hinge_offset=b["l1"], mass=b["mass"], cg_offset=b["l2"])
        elif b["kind"] == "torsional":
            c.add_torsional(b["hinge"], b["theta0"], b["n_pts"], w["ds"], b["inertia"], b["damping"], b["stiffness"],
                            b["theta"])
        elif b["kind"] == "deformable":
            c.add_deformable(b["clamp"], b["theta0"], b["n_pts"], w["ds"], b["mass"], b["ei"], b["ea"], b["tip_angle"])
        else:
            c.add_rigid(b["pts"], w["ds"], b.get("ur"), b.get("appended", False))
    if w.get("sd_box") is not None:
        if np.ndim(w["sd_box"]) == 2:      # a union of boxes
            c.set_subdomain_boxes(w["sd_box"])
        else:
            c.set_subdomain(*w["sd_box"])
        if precompute:
            c.precompute(drop_tol)
    return c


def oracle_history(sim, body=0):
    return np.array([[r["bodies"][body][k] for k in ("fx", "fy", "moment", "theta", "phi")] + [r["iters"]]
                     for r in sim.history])


def rel_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def check_rel(tag, got, ref, tol):
    """Assert rel_err(got, ref) < tol and print the measured error (tag) for the record."""
    err = rel_err(got, ref)
    print("PARITY %s rel %.3e (bound %.0e)" % (tag, err, tol))
    assert err < tol, (tag, err)
    return err
