// Kernel tables of the row-block executor for one element type (one translation unit per
// type, so that the two compile in parallel).
#pragma once

#include "sf_block.cuh"
#include "sf_block_ws.cuh"
#include "sf_block_tma.cuh"

namespace sf {

template <int MODE, typename T>
const void *block_kernel_lpr(int lpr) {
    switch (lpr) {
        case 1: return (const void *)k_block_exec<MODE, T, 1>;
        case 2: return (const void *)k_block_exec<MODE, T, 2>;
        case 4: return (const void *)k_block_exec<MODE, T, 4>;
        case 32: return (const void *)k_block_exec<MODE, T, 32>;
        default: return nullptr;
    }
}

// Warp-specialised row-block kernel of a mode.
template <typename T>
const void *block_ws_kernel_t(int mode) {
    switch (mode) {
        case M_TRSV_SPMV: return (const void *)k_block_ws<M_TRSV_SPMV, T>;
        case M_TRSV: return (const void *)k_block_ws<M_TRSV, T>;
        case M_SPMV_TRSV: return (const void *)k_block_ws<M_SPMV_TRSV, T>;
        case M_ADJ_TRSV_SPMV: return (const void *)k_block_ws<M_ADJ_TRSV_SPMV, T>;
        case M_ADJ_SPMV_TRSV: return (const void *)k_block_ws<M_ADJ_SPMV_TRSV, T>;
        default: return nullptr;
    }
}

// Packed-record row-block kernel (which = 0) or its value-packing pre-pass (which = 1).
template <typename T>
const void *block_tma_kernel_t(int mode, int which) {
    switch (mode) {
        case M_TRSV_SPMV: return which ? (const void *)k_pack_vals<M_TRSV_SPMV, T> : (const void *)k_block_tma<M_TRSV_SPMV, T>;
        case M_TRSV: return which ? (const void *)k_pack_vals<M_TRSV, T> : (const void *)k_block_tma<M_TRSV, T>;
        case M_SPMV_TRSV: return which ? (const void *)k_pack_vals<M_SPMV_TRSV, T> : (const void *)k_block_tma<M_SPMV_TRSV, T>;
        case M_ADJ_TRSV_SPMV:
            return which ? (const void *)k_pack_vals<M_ADJ_TRSV_SPMV, T> : (const void *)k_block_tma<M_ADJ_TRSV_SPMV, T>;
        case M_ADJ_SPMV_TRSV:
            return which ? (const void *)k_pack_vals<M_ADJ_SPMV_TRSV, T> : (const void *)k_block_tma<M_ADJ_SPMV_TRSV, T>;
        default: return nullptr;
    }
}

// lpr == 0 selects the pre-pass of the mode.
template <typename T>
const void *block_kernel_t(int mode, int lpr) {
    switch (mode) {
        case M_TRSV_SPMV: return lpr ? block_kernel_lpr<M_TRSV_SPMV, T>(lpr) : (const void *)k_block_prep<M_TRSV_SPMV, T>;
        case M_TRSV: return lpr ? block_kernel_lpr<M_TRSV, T>(lpr) : (const void *)k_block_prep<M_TRSV, T>;
        case M_SPMV_TRSV: return lpr ? block_kernel_lpr<M_SPMV_TRSV, T>(lpr) : (const void *)k_block_prep<M_SPMV_TRSV, T>;
        case M_ADJ_TRSV_SPMV:
            return lpr ? block_kernel_lpr<M_ADJ_TRSV_SPMV, T>(lpr) : (const void *)k_block_prep<M_ADJ_TRSV_SPMV, T>;
        case M_ADJ_SPMV_TRSV:
            return lpr ? block_kernel_lpr<M_ADJ_SPMV_TRSV, T>(lpr) : (const void *)k_block_prep<M_ADJ_SPMV_TRSV, T>;
        default: return nullptr;
    }
}

const void *block_kernel_f64(int mode, int lpr);
const void *block_kernel_f32(int mode, int lpr);
const void *block_ws_kernel_f64(int mode);
const void *block_ws_kernel_f32(int mode);
const void *block_tma_kernel_f64(int mode, int which);
const void *block_tma_kernel_f32(int mode, int which);

}  // namespace sf
