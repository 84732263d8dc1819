// Root conversion helpers shared by the tree engines: the FP64 packed root
// (real or complex entries) converted to the element type of a variant.
#pragma once
#include <algorithm>
#include <string>

#include "gbs_internal.h"
#include "gbs_tree.cuh"

namespace gbs {

template <class E> struct root_src { typedef double type; };
template <class T> struct root_src<cplx<T>> { typedef cplx<double> type; };

template <class E> GBS_HD E conv_entry(const typename root_src<E>::type& x);
template <> GBS_HD double conv_entry<double>(const double& x) { return x; }
template <> GBS_HD float conv_entry<float>(const double& x) { return (float)x; }
template <> GBS_HD dd conv_entry<dd>(const double& x) { return dd_make(x); }
template <> GBS_HD td conv_entry<td>(const double& x) { return td_make(x); }
template <> GBS_HD cplx<double> conv_entry<cplx<double>>(const cplx<double>& x) { return x; }
template <> GBS_HD cplx<float> conv_entry<cplx<float>>(const cplx<double>& x) { return {(float)x.re, (float)x.im}; }
template <> GBS_HD cplx<dd> conv_entry<cplx<dd>>(const cplx<double>& x) { return {dd_make(x.re), dd_make(x.im)}; }
template <> GBS_HD cplx<td> conv_entry<cplx<td>>(const cplx<double>& x) { return {td_make(x.re), td_make(x.im)}; }

}  // namespace gbs
