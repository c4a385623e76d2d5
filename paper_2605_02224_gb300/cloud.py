"""Cloud: an owning Python handle around one mknn_cloud (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import mknn as M


class Cloud:
    """Owns a built cloud; frees it when closed or collected."""

    def __init__(self, handle: int):
        self.handle = handle
        self.n, self.E, _ = M.mknn_cloud_info(handle)

    @classmethod
    def build(cls, xyz, order=None, keep_tets: bool = False, dynamic: bool = False) -> "Cloud":
        return cls(M.mknn_build(xyz, order, keep_tets, dynamic))

    @classmethod
    def from_table(cls, xyz_ranked, rowp, succ) -> "Cloud":
        return cls(M.mknn_cloud_from_table(xyz_ranked, rowp, succ))

    @classmethod
    def load(cls, path: str) -> "Cloud":
        return cls(M.mknn_cloud_load(path))

    def save(self, path: str):
        M.mknn_cloud_save(self.handle, path)

    def append(self, xyz, stream: int = 0) -> "Cloud":
        """Inserts points after the existing ones (dynamic clouds)."""
        M.mknn_cloud_append(self.handle, xyz, stream)
        return self

    def compact(self, stream: int = 0) -> "Cloud":
        """Lays a dynamic cloud's device table out afresh."""
        M.mknn_cloud_compact(self.handle, stream)
        return self

    def upload(self, stream: int = 0) -> "Cloud":
        M.mknn_cloud_upload(self.handle, stream)
        return self

    def table(self):
        return M.mknn_cloud_table(self.handle)

    def order(self) -> np.ndarray:
        return M.mknn_cloud_order(self.handle)

    def stats(self) -> dict:
        return M.mknn_cloud_stats(self.handle)

    def tets(self) -> np.ndarray:
        return M.mknn_cloud_tets(self.handle)

    def device_bytes(self) -> int:
        return M.mknn_cloud_info(self.handle)[2]

    def trees(self):
        """(box trees on the device copy, entries of the lists they cover)."""
        return M.mknn_cloud_trees(self.handle)

    def knn(self, q, k: int, m=None, stream: int = 0, **opt):
        """q: torch CUDA tensor (nq, 3 or 4) float32; m: None, int or int32
        CUDA tensor (nq,). Returns (idx int32 (nq,k), d2 float32 (nq,k))."""
        import torch
        nq = int(q.shape[0])
        idx = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        if stream == 0:
            stream = torch.cuda.current_stream(q.device).cuda_stream
        m_ptr, m_scalar = (None, int(m or 0)) if (m is None or isinstance(m, int)) else (m, 0)
        if opt:
            M.mknn_knn_ex(self.handle, q, nq, int(q.stride(0)), k, m_ptr, m_scalar, idx, d2,
                          stream, **opt)
        else:
            M.mknn_knn(self.handle, q, nq, int(q.stride(0)), k, m_ptr, m_scalar, idx, d2, stream)
        return idx, d2

    def knn_sites(self, sites, k: int, m=None, stream: int = 0, **opt):
        """sites: int32 CUDA tensor (nq,) of ranks; query i is that site.
        Returns (idx int32 (nq,k), d2 float32 (nq,k))."""
        import torch
        nq = int(sites.shape[0])
        idx = torch.empty((nq, k), dtype=torch.int32, device=sites.device)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=sites.device)
        if stream == 0:
            stream = torch.cuda.current_stream(sites.device).cuda_stream
        m_ptr, m_scalar = (None, int(m or 0)) if (m is None or isinstance(m, int)) else (m, 0)
        M.mknn_knn_sites(self.handle, sites, nq, k, m_ptr, m_scalar, idx, d2, stream, **opt)
        return idx, d2

    def knn_host(self, q, k: int, m=None, out_idx=None, out_d2=None):
        m_arr, m_scalar = (None, int(m or 0)) if (m is None or isinstance(m, int)) else (m, 0)
        return M.mknn_knn_host(self.handle, q, k, m_arr, m_scalar, out_idx, out_d2)

    def check(self) -> int:
        return M.mknn_cloud_check(self.handle)

    def close(self):
        if self.handle:
            M.mknn_cloud_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
