"""Convenience layer over the C ABI: geometry registration from mesh/SDF descriptions
and torch-tensor calls of the forward manifold.  Argument marshalling only."""
from __future__ import annotations

import numpy as np
import torch

from . import api


class Engine:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.ctx = api.cm_create_context(device, hbm_budget_bytes)

    def close(self):
        if self.ctx is not None:
            api.cm_destroy_context(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_geometry(self, g) -> int:
        """Registers an object with kind, dims, verts (V, 4), edges (E, 2), planes (F, 4)."""
        return api.cm_create_geometry(self.ctx, g.kind, g.dims, g.verts, g.edges,
                                      g.planes if len(g.planes) else None)

    def add_hull(self, points) -> int:
        """Registers the convex hull of ``points`` ((n, 3)), built by the library."""
        return api.cm_create_hull_geometry(self.ctx, points)

    def add_primitive(self, kind, dims, tess=0) -> int:
        """Registers a primitive whose mesh the library generates (resolution ``tess``)."""
        return api.cm_create_primitive_geometry(self.ctx, kind, dims, tess)

    def add_geometries(self, geoms) -> np.ndarray:
        ids = np.array([self.add_geometry(g) for g in geoms], dtype=np.int32)
        api.cm_sync_geometry(self.ctx)
        return ids

    def params(self, **kw) -> api.cm_params:
        return api.cm_default_params(**kw)

    def forward(self, pair_geoms, poses, dims=None, tau=None, params=None, out=None, stream=None):
        params = params or self.params()
        n = int(pair_geoms.shape[0])
        if out is None:
            out = torch.empty((n, params.K, 8), dtype=torch.float32, device=pair_geoms.device)
        api.cm_contact_manifold_fwd(self.ctx, pair_geoms, poses, dims, tau, params, out, stream)
        return out

    def forward_dump(self, pair_geoms, poses, dims=None, tau=None, params=None, stream=None):
        """(out, candidates, offsets): the forward manifold, every candidate row (rows, 8) in
        world coordinates and the host offsets (n + 1) of each pair's first row."""
        params = params or self.params()
        n = int(pair_geoms.shape[0])
        off = api.cm_candidate_offsets(self.ctx, pair_geoms.cpu().numpy(), params)
        out = torch.empty((n, params.K, 8), dtype=torch.float32, device=pair_geoms.device)
        cand = torch.empty((max(int(off[-1]), 1), 8), dtype=torch.float32, device=pair_geoms.device)
        d_off = torch.as_tensor(off, device=pair_geoms.device)
        api.cm_contact_manifold_fwd_dump(self.ctx, pair_geoms, poses, dims, tau, params, out, cand, d_off, stream)
        return out, cand, off

    def forward_save(self, pair_geoms, poses, dims=None, tau=None, params=None, stream=None):
        """(out, saved): the forward manifold and each pair's record for ``backward``."""
        params = params or self.params()
        n = int(pair_geoms.shape[0])
        out = torch.empty((n, params.K, 8), dtype=torch.float32, device=pair_geoms.device)
        saved = torch.empty((n, api.cm_saved_stride(self.ctx, params)), dtype=torch.float32,
                            device=pair_geoms.device)
        api.cm_contact_manifold_fwd_save(self.ctx, pair_geoms, poses, dims, tau, params, out, saved, stream)
        return out, saved

    def backward(self, pair_geoms, poses, dims, tau, grad_out, params=None, stream=None, saved=None):
        """(dL/d poses, dL/d dims or None) for upstream ``grad_out`` (n, K, 8); from the
        forward's records when ``saved`` (see ``forward_save``) is given, else recomputing
        the forward."""
        params = params or self.params()
        gp = torch.empty_like(poses)
        gd = None if dims is None else torch.empty_like(dims)
        if saved is None:
            api.cm_contact_manifold_bwd(self.ctx, pair_geoms, poses, dims, tau, params,
                                        grad_out.contiguous(), gp, gd, stream)
        else:
            api.cm_contact_manifold_bwd_saved(self.ctx, pair_geoms, poses, dims, tau, params, saved,
                                              grad_out.contiguous(), gp, gd, stream)
        return gp, gd

    def check(self):
        api.cm_check_device_error(self.ctx)


class ContactManifold(torch.autograd.Function):
    """out = manifold(poses, dims); differentiable in poses and dims through the
    library's adjoint kernel (the forward keeps each pair's per-pair reductions, the
    backward recomputes every candidate from them)."""

    @staticmethod
    def forward(ctx, poses, dims, engine, pair_geoms, tau, params):
        out, saved = engine.forward_save(pair_geoms, poses.detach().contiguous(),
                                         None if dims is None else dims.detach().contiguous(), tau, params)
        ctx.engine, ctx.params = engine, params
        ctx.has_dims = dims is not None
        ctx.save_for_backward(poses.detach(), dims.detach() if dims is not None else poses.new_empty(0),
                              pair_geoms, tau if tau is not None else poses.new_empty(0), saved)
        ctx.has_tau = tau is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        poses, dims, pg, tau, saved = ctx.saved_tensors
        gp, gd = ctx.engine.backward(pg, poses.contiguous(), dims.contiguous() if ctx.has_dims else None,
                                     tau if ctx.has_tau else None, grad_out, ctx.params, saved=saved)
        return gp, (gd if ctx.has_dims else None), None, None, None, None


def contact_manifold(engine, pair_geoms, poses, dims=None, tau=None, params=None):
    """Differentiable manifold (n, K, 8) of the pairs; see ``ContactManifold``."""
    return ContactManifold.apply(poses, dims, engine, pair_geoms, tau, params or engine.params())


def workload_tensors(w, device="cuda", id_map=None):
    """Device tensors (pair_geoms, poses, dims, tau) of a synthetic workload."""
    pg = w.pair_geoms if id_map is None else id_map[w.pair_geoms]
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)  # noqa: E731
    return (t(pg, torch.int32), t(w.poses, torch.float32), t(w.dims, torch.float32),
            t(w.tau, torch.float32))
