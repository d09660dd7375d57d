// tables.h -- 1-D reference tables of the nodal RT_k x Q_k basis (host side).
#pragma once
#include "device.cuh"

namespace mgd {
// Fills the tables of degree K in double and float (computed in double).
template <int K> void make_tables(Tab<K, double>& td, Tab<K, float>& tf);
}  // namespace mgd
